"""Seeded synthetic inputs shared by the oracle and the CUDA path (no method arithmetic)."""
from .workloads import *  # noqa: F401,F403
from .small import *  # noqa: F401,F403

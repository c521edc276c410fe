"""Shared helpers of the GPU parity tests: workload set-up from the seeded
generator, the FP64 oracle beside the CUDA path, and the tolerance checks.

Tolerances (relative 1e-5 against FP64, with floors where a value can be 0):
  CV      |ds_d|      <= 1e-5 |s_d|
  bias    |dV|        <= 1e-5 max(|V|, w0)
  dV/ds   |d(dV/ds)|  <= 1e-5 max(|dV/ds_d|, w0 / sigma_d)
  forces  ||dF||_2 / ||F||_2 <= 1e-5  and  max_i |dF_i| <= 1e-5 max_i |F_i|
"""
import numpy as np

import oracle
import synth

TOL = 1e-5


def kbdt(mp):
    return mp.kB * mp.temperature * (mp.biasfactor - 1.0)


def check_cv(s_gpu, s_ref, tol=TOL):
    s_gpu, s_ref = np.asarray(s_gpu), np.asarray(s_ref)
    assert np.all(np.abs(s_gpu - s_ref) <= tol * np.abs(s_ref)), (s_gpu, s_ref, (s_gpu - s_ref) / s_ref)


def check_bias(V, dV, V_ref, dV_ref, mp, tol=TOL):
    assert abs(V - V_ref) <= tol * max(abs(V_ref), mp.w0), (V, V_ref)
    for d in range(len(dV_ref)):
        floor = mp.w0 / mp.sigma[d]
        assert abs(dV[d] - dV_ref[d]) <= tol * max(abs(dV_ref[d]), floor), (d, dV, dV_ref)


def force_errors(F, F_ref):
    F = np.asarray(F, dtype=np.float64)
    nrm = np.linalg.norm(F - F_ref) / max(np.linalg.norm(F_ref), 1e-300)
    per = np.max(np.linalg.norm(F - F_ref, axis=1)) / max(np.max(np.linalg.norm(F_ref, axis=1)), 1e-300)
    return nrm, per


def check_forces(F, F_ref, tol=TOL):
    nrm, per = force_errors(F, F_ref)
    assert nrm <= tol and per <= tol, (nrm, per)
    return nrm, per


def setup_hills(system, mp, count, cfg, base_frame=None):
    """Hill centres uniform in s_ref +- 10 sigma, s_ref the oracle CV of the
    unperturbed base frame, and their oracle well-tempered heights."""
    p = oracle.params_from(mp, system.box)
    s_ref, _, _ = oracle.cv(system.base if base_frame is None else base_frame, p)
    c = synth.hill_centres(cfg, system.sys, s_ref, mp.sigma, count)
    return c, s_ref

"""Seeded synthetic workloads for the metadynamics bias path.

This module is shared by the FP64 oracle and the CUDA path as their only
common input source, so it holds no arithmetic of the method itself (no
switching function, no spherical harmonics, no hills, no bias): it builds
atom positions, species, perturbation frames, uniform hill centres and
request traces, all from ``numpy.random.SeedSequence(6873, spawn_key=...)``
with PCG64, plus a small C routine (``rsa.c``) for random sequential
addition of hard-core liquid atoms.

Frames are float32 ``[N, 4]`` arrays: x, y, z in Angstrom, already wrapped
into ``[0, L)``, and the species id (0 or 1) stored as a float in column 3.

The workload shapes stand in for the GaN systems of the paper's large-scale
runs (B4 wurtzite, 27,648 to 2.2 M atoms; Section "B4-B1 phase transition in
Large-scale systems") and its size sweep (50 k to 1.3 M atoms; Section
"Efficiency of GPU-MetaD package"); the paper's datasets and trajectories are
not used.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_rsa.so")
_ROOT_SEED = 6873

# ---------------------------------------------------------------- constants
# Method parameters of the five workloads.  They are plain numbers handed to
# both implementations; nothing here evaluates them.
KB_KJMOL = 0.0083144626  # Boltzmann constant in kJ/mol/K
WURTZITE_A = 3.19
WURTZITE_C = 5.19
WURTZITE_U = 3.0 / 8.0
LIQUID_DENSITY = 0.08  # atoms / A^3


@dataclass
class MethodParams:
    """Switch, CV and bias parameters shared by every workload."""
    rc: float = 3.5
    r0: float = 2.5
    sw_n: int = 6
    sw_m: int = 12
    cn_unlike_only: bool = True
    n_cv: int = 2
    sigma: tuple = (0.05, 0.02)
    w0: float = 1.0
    biasfactor: float = 10.0
    temperature: float = 300.0
    kB: float = KB_KJMOL


@dataclass
class System:
    """One periodic system: base frame (float32 [N,4]) and box lengths."""
    base: np.ndarray
    box: np.ndarray  # float64 [3]
    cfg: int
    sys: int
    info: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.base.shape[0])


# ---------------------------------------------------------------- seeding
def seed_sequence(cfg: int, sys: int, *key: int) -> np.random.SeedSequence:
    return np.random.SeedSequence(_ROOT_SEED, spawn_key=(int(cfg), int(sys)) + tuple(int(k) for k in key))


def rng(cfg: int, sys: int, *key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_sequence(cfg, sys, *key)))


# ---------------------------------------------------------------- native RSA
_lib = None


def build_native(force: bool = False) -> str:
    """Compile rsa.c into synth/_rsa.so with plain IEEE double arithmetic."""
    src = os.path.join(_HERE, "rsa.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _rsa_lib():
    global _lib
    if _lib is None:
        build_native()
        lib = ctypes.CDLL(_SO)
        lib.synth_rsa_fill.restype = ctypes.c_int
        lib.synth_rsa_fill.argtypes = [
            ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64,
            ctypes.POINTER(ctypes.c_int64)]
        _lib = lib
    return _lib


def rsa_fill(existing_xyz: np.ndarray, n_new: int, box, xlo: float, xhi: float, dmin: float,
             seed: int, max_attempts: int | None = None) -> np.ndarray:
    """Place n_new hard-core points in x in [xlo, xhi) avoiding existing atoms."""
    lib = _rsa_lib()
    ex = np.ascontiguousarray(existing_xyz, dtype=np.float32).reshape(-1, 3)
    out = np.zeros((n_new, 3), dtype=np.float32)
    b = np.ascontiguousarray(box, dtype=np.float64)
    if max_attempts is None:
        max_attempts = 4000 * max(n_new, 1) + 10_000_000
    att = ctypes.c_int64(0)
    rc = lib.synth_rsa_fill(ex.shape[0], ex.ctypes.data, n_new, out.ctypes.data, b.ctypes.data,
                            float(xlo), float(xhi), float(dmin), ctypes.c_uint64(seed & (2**64 - 1)),
                            int(max_attempts), ctypes.byref(att))
    if rc == -2:
        raise RuntimeError(f"RSA jammed: placed fewer than {n_new} points in {att.value} attempts")
    if rc != 0:
        raise RuntimeError(f"synth_rsa_fill failed with code {rc}")
    return out


# ---------------------------------------------------------------- wrapping
def wrap_to_box(x64: np.ndarray, box) -> np.ndarray:
    """Wrap FP64 coordinates into [0, L): x - L*floor(x/L), rounded to
    float32; a coordinate that rounds up to L becomes 0."""
    box = np.asarray(box, dtype=np.float64)
    w = x64 - box * np.floor(x64 / box)
    f = w.astype(np.float32)
    f = np.where(f.astype(np.float64) >= box, np.float32(0.0), f)
    return f.astype(np.float32)


# ---------------------------------------------------------------- builders
def rsa_liquid_system(n: int, density: float, dmin: float, cfg: int, sys: int) -> System:
    """Cubic box at the given density filled by RSA, species 50/50 shuffled."""
    L = (n / density) ** (1.0 / 3.0)
    box = np.array([L, L, L], dtype=np.float64)
    ss = seed_sequence(cfg, sys, 0).spawn(3)
    seed = int(ss[0].generate_state(1, dtype=np.uint64)[0])
    xyz = rsa_fill(np.zeros((0, 3), np.float32), n, box, 0.0, L, dmin, seed)
    species = np.zeros(n, dtype=np.float32)
    species[n // 2:] = 1.0
    species = np.random.Generator(np.random.PCG64(ss[1])).permutation(species)
    base = np.concatenate([xyz, species[:, None]], axis=1).astype(np.float32)
    return System(base=np.ascontiguousarray(base), box=box, cfg=cfg, sys=sys,
                  info={"kind": "rsa_liquid", "density": density, "dmin": dmin})


def wurtzite_cell(a: float, c: float, u: float):
    """Orthorhombic a x sqrt(3)a x c wurtzite cell: 8 atoms (4 of each species),
    fractional coordinates and species ids."""
    fa = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 1.0 / 6.0, 0.5], [0.0, 2.0 / 3.0, 0.5]])
    fb = fa + np.array([0.0, 0.0, u])
    frac = np.concatenate([fa, fb]) % 1.0
    spec = np.array([0, 0, 0, 0, 1, 1, 1, 1], dtype=np.float32)
    dims = np.array([a, math.sqrt(3.0) * a, c])
    return frac, spec, dims


def wurtzite_liquid_system(n: int, cfg: int, sys: int, density_scale: float = 1.0,
                           lattice_noise: float = 0.1, liquid_dmin: float = 2.0,
                           liquid_density: float = LIQUID_DENSITY) -> System:
    """Wurtzite-like lattice slab with N(0, noise) displacements (about half
    the box, x < half*a) and an RSA liquid slab at liquid_density beside it
    (min distance dmin to every atom, lattice included); exactly n atoms.  A
    density_scale j rescales every length by j**(-1/3)."""
    lf = density_scale ** (-1.0 / 3.0)
    a, c = WURTZITE_A * lf, WURTZITE_C * lf
    noise = lattice_noise * lf
    dmin = liquid_dmin * lf
    rho_liq = liquid_density * density_scale
    frac, spec, dims = wurtzite_cell(a, c, WURTZITE_U)
    rho_lat = 8.0 / float(np.prod(dims))
    L = (n / (0.5 * (rho_lat + rho_liq))) ** (1.0 / 3.0)
    half = max(1, int(round(L / (2 * dims[0]))))
    ny = max(1, int(round(L / dims[1])))
    nz = max(1, int(round(L / dims[2])))
    while half > 1 and 8 * half * ny * nz >= n:
        half -= 1
    n_lat0 = 8 * half * ny * nz
    if n_lat0 >= n:
        raise ValueError(f"{n} atoms is too few for a lattice slab")
    # the liquid slab is as wide as its atom count needs at density rho_liq
    lx_liq = (n - n_lat0) / (rho_liq * ny * dims[1] * nz * dims[2])
    box = np.array([half * dims[0] + lx_liq, ny * dims[1], nz * dims[2]], dtype=np.float64)
    ix, iy, iz = np.meshgrid(np.arange(half), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    lat = ((cells[:, None, :] + frac[None, :, :]) * dims[None, None, :]).reshape(-1, 3)
    lat_spec = np.tile(spec, cells.shape[0])
    n_lat = lat.shape[0]
    n_liq = n - n_lat
    if n_liq < 0:
        raise ValueError(f"lattice alone holds {n_lat} > {n} atoms")
    ss = seed_sequence(cfg, sys, 0).spawn(4)
    g_noise = np.random.Generator(np.random.PCG64(ss[0]))
    lat = wrap_to_box(lat + g_noise.normal(0.0, noise, size=lat.shape), box)
    seed = int(ss[1].generate_state(1, dtype=np.uint64)[0])
    liq = rsa_fill(lat, n_liq, box, half * dims[0], box[0], dmin, seed)
    liq_spec = np.zeros(n_liq, dtype=np.float32)
    liq_spec[n_liq // 2:] = 1.0
    liq_spec = np.random.Generator(np.random.PCG64(ss[2])).permutation(liq_spec)
    xyz = np.concatenate([lat, liq]).astype(np.float32)
    species = np.concatenate([lat_spec, liq_spec]).astype(np.float32)
    order = np.random.Generator(np.random.PCG64(ss[3])).permutation(n)
    base = np.concatenate([xyz[order], species[order, None]], axis=1).astype(np.float32)
    return System(base=np.ascontiguousarray(base), box=box, cfg=cfg, sys=sys,
                  info={"kind": "wurtzite_liquid", "n_lattice": int(n_lat), "n_liquid": int(n_liq),
                        "liquid_density": n_liq / ((box[0] - half * dims[0]) * box[1] * box[2]),
                        "density_scale": density_scale, "cells": [half, ny, nz]})


def perturbed_frame(system: System, frame: int, sigma: float = 0.05) -> np.ndarray:
    """Frame f = wrap(base + eps_f), eps_f ~ N(0, sigma^2) iid per coordinate,
    independent per frame (not cumulative)."""
    g = rng(system.cfg, system.sys, 1, frame)
    eps = g.normal(0.0, sigma, size=(system.n, 3))
    xyz = wrap_to_box(system.base[:, :3].astype(np.float64) + eps, system.box)
    out = np.empty_like(system.base)
    out[:, :3] = xyz
    out[:, 3] = system.base[:, 3]
    return out


def drift_trajectory(system: System, count: int, step_sigma: float = 0.01, sigma: float = 0.05):
    """Frames 0 .. count-1 of a drifting trajectory, in order: frame f =
    wrap(base + W_f + eps_f), where W_f = sum_{t=1..f} xi_t is a per-atom
    random walk (xi_t ~ N(0, step_sigma^2) iid per coordinate and frame,
    W_0 = 0) and eps_f the thermal noise of perturbed_frame (so frame 0 is
    perturbed_frame(system, 0)).  Atoms leave their neighbour shells at a
    molecular-dynamics-like rate, so a Verlet list is rebuilt every few tens
    of frames.  Yields float32 [N, 4] arrays."""
    walk = np.zeros((system.n, 3))
    for f in range(count):
        if f > 0:
            walk += rng(system.cfg, system.sys, 7, f).normal(0.0, step_sigma, size=(system.n, 3))
        eps = rng(system.cfg, system.sys, 1, f).normal(0.0, sigma, size=(system.n, 3))
        out = np.empty_like(system.base)
        out[:, :3] = wrap_to_box(system.base[:, :3].astype(np.float64) + walk + eps, system.box)
        out[:, 3] = system.base[:, 3]
        yield out


def hill_centres(cfg: int, sys: int, centre, sigma, count: int, half_width_sigmas: float = 10.0) -> np.ndarray:
    """Hill centres uniform in prod_d [centre_d - 10 sigma_d, centre_d + 10 sigma_d]."""
    centre = np.atleast_1d(np.asarray(centre, dtype=np.float64))
    sigma = np.atleast_1d(np.asarray(sigma, dtype=np.float64))[: centre.size]
    u = rng(cfg, sys, 2).random((count, centre.size))
    lo = centre - half_width_sigmas * sigma
    return lo + u * (2.0 * half_width_sigmas * sigma)


# ---------------------------------------------------------------- configs
def _cache_dir() -> str:
    d = os.environ.get("METAD_SYNTH_CACHE", os.path.join(tempfile.gettempdir(), "metad_synth_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key: str, make):
    h = hashlib.sha1(key.encode()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"sys_{h}.npz")
    if os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        info = dict(zip(z["info_k"].tolist(), z["info_v"].tolist())) if "info_k" in z else {}
        return System(base=z["base"], box=z["box"], cfg=int(z["cfg"]), sys=int(z["sys"]), info=info)
    s = make()
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, base=s.base, box=s.box, cfg=s.cfg, sys=s.sys,
             info_k=np.array([str(k) for k in s.info]), info_v=np.array([str(v) for v in s.info.values()]))
    os.replace(tmp, path)
    return s


def config1_system() -> System:
    """1,000 atoms, cubic box at 0.08 atoms/A^3, RSA at 1.8 A, 50/50 species."""
    return _cached("cfg1-v1", lambda: rsa_liquid_system(1000, LIQUID_DENSITY, 1.8, cfg=1, sys=0))


def wurtzite_system(n: int, cfg: int, sys: int = 0, density_scale: float = 1.0) -> System:
    return _cached(f"wl-v2-{n}-{cfg}-{sys}-{density_scale!r}",
                   lambda: wurtzite_liquid_system(n, cfg, sys, density_scale=density_scale))


def config2_system() -> System:
    return wurtzite_system(100_000, cfg=2)


def config3_system() -> System:
    return wurtzite_system(1_000_000, cfg=3)


CONFIG_PARAMS = {
    1: dict(n_cv=1, sigma=(0.05,), hills=200, frames=100, fp64=True),
    2: dict(n_cv=2, sigma=(0.05, 0.02), hills=5000, frames=100, fp64=False),
    3: dict(n_cv=2, sigma=(0.05, 0.02), hills_folded=20000, hills=20000, frames=10000,
            deposit_every=500, grid_n=(200, 200), fp64=False),
    4: dict(n_cv=2, sigma=(0.05, 0.02), systems=64, steps=10, fp64=False),
    5: dict(n_cv=2, sigma=(0.05, 0.02), walkers=32, requests=2000, rate_hz=5000.0, hills=1000,
            deposit_every=20, budget_bytes=120 * 10**9, fp64=False),
}


def method_params(cfg: int) -> MethodParams:
    p = CONFIG_PARAMS.get(cfg, CONFIG_PARAMS[2])
    return MethodParams(n_cv=p["n_cv"], sigma=tuple(p["sigma"]))


def batch_layout(cfg: int = 4, n_systems: int = 64, n_lo: float = 1e3, n_hi: float = 2e5,
                 k_lo: float = 100, k_hi: float = 1e4):
    """Atom counts and hill counts log-uniform, density factor U(0.9, 1.1)."""
    g = rng(cfg, 0, 3)
    n = np.round(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), n_systems))).astype(np.int64)
    k = np.round(np.exp(g.uniform(math.log(k_lo), math.log(k_hi), n_systems))).astype(np.int64)
    dens = g.uniform(0.9, 1.1, n_systems)
    return n, k, dens


def served_trace(cfg: int = 5, n_walkers: int = 32, n_requests: int = 2000, rate_hz: float = 5000.0,
                 n_lo: float = 2e3, n_hi: float = 5e5):
    """Walker atom counts log-uniform; Poisson arrivals (exponential gaps);
    the walker of each request uniform."""
    g = rng(cfg, 0, 4)
    n = np.round(np.exp(g.uniform(math.log(n_lo), math.log(n_hi), n_walkers))).astype(np.int64)
    gaps = g.exponential(1.0 / rate_hz, n_requests)
    arrivals = np.cumsum(gaps)
    walker = g.integers(0, n_walkers, n_requests)
    return n, arrivals, walker


def served_arrivals(cfg: int, n_walkers: int, n_requests: int, rate_hz: float, seed: int):
    """Another request stream for the walkers of served_trace: Poisson
    arrivals at rate_hz (all at t = 0 when rate_hz is infinite: a saturating
    burst) and uniform walkers, from seed `seed` (>= 1; the walker sizes are
    served_trace's)."""
    g = rng(cfg, seed, 8)
    if math.isinf(rate_hz):
        arrivals = np.zeros(n_requests)
    else:
        arrivals = np.cumsum(g.exponential(1.0 / rate_hz, n_requests))
    walker = g.integers(0, n_walkers, n_requests)
    return arrivals, walker


def npt_frame(system: System, frame: int, strain_sigma: float = 1e-3, sigma: float = 0.05, period: int = 0):
    """A frame of a triaxial NPT run: each box length scaled by 1 + e_a,
    positions scaled with it (fixed fractional coordinates) plus N(0, sigma^2)
    noise, wrapped into the new box.  e_a ~ N(0, strain_sigma^2)
    independently per axis and frame, or with period > 0 a slow oscillation
    e_a = strain_sigma sin(2 pi frame / period + phi_a) (phases fixed per
    system), as a barostat moves the box.  Returns (float32 [N, 4] frame,
    float64 [3] box)."""
    g = rng(system.cfg, system.sys, 5, frame)
    if period > 0:
        phi = 2.0 * math.pi * rng(system.cfg, system.sys, 6).random(3)
        e = strain_sigma * np.sin(2.0 * math.pi * frame / period + phi)
        g.normal(0.0, strain_sigma, size=3)  # keep the noise stream of the iid form
    else:
        e = g.normal(0.0, strain_sigma, size=3)
    box = system.box * (1.0 + e)
    eps = g.normal(0.0, sigma, size=(system.n, 3))
    xyz = wrap_to_box(system.base[:, :3].astype(np.float64) * (1.0 + e) + eps, box)
    out = np.empty_like(system.base)
    out[:, :3] = xyz
    out[:, 3] = system.base[:, 3]
    return out, box

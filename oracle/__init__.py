"""FP64 CPU oracle for the metadynamics bias path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library path never does; it shares no code with the CUDA implementation.

The arithmetic lives in ``metad_oracle.c`` (plain IEEE double, no fused
multiply-add); this module compiles it with gcc and marshals numpy arrays.
Every function states the definition it follows; the readings taken where
the paper is silent are listed in ``metad_oracle.c`` beside each function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "metad_oracle.c")
_SO = os.path.join(_HERE, "_metad_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("rc", ctypes.c_double), ("r0", ctypes.c_double),
                ("sw_n", ctypes.c_int32), ("sw_m", ctypes.c_int32), ("stretch", ctypes.c_int32),
                ("cn_unlike_only", ctypes.c_int32), ("n_cv", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 2), ("pad", ctypes.c_int32 * 2), ("lo", ctypes.c_double * 2),
                ("hi", ctypes.c_double * 2), ("data", ctypes.c_void_p)]


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "orc_pairs_brute": (I64, [I32, P, P, D, P, I64]),
            "orc_pairs_cells": (I64, [I32, P, P, D, P, I64, ctypes.c_int]),
            "orc_switch": (None, [P, I32, P, P, P]),
            "orc_ylm": (None, [I32, P, P, P, P, P]),
            "orc_cv": (ctypes.c_int, [I32, P, P, P, P, P, ctypes.c_int]),
            "orc_forces": (ctypes.c_int, [I32, P, P, P, P, P, ctypes.c_int]),
            "orc_grid_fold": (ctypes.c_int, [P, I32, P, P, P, ctypes.c_int]),
            "orc_bias": (ctypes.c_int, [I32, P, I32, P, P, P, P, P, P, P]),
            "orc_deposit_sequence": (ctypes.c_int, [I32, I32, I32, P, P, P, P, D, D, P]),
            "orc_step": (ctypes.c_int, [I32, P, P, I32, P, P, P, P, P, P, P, P, ctypes.c_int]),
            "orc_max_threads": (ctypes.c_int, []),
            "orc_step_box": (ctypes.c_int, [I32, P, P, I32, I32, P, P, P, P, P, P, P, P, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_L().orc_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f32x4(pos4):
    a = np.ascontiguousarray(pos4, dtype=np.float32)
    assert a.ndim == 2 and a.shape[1] == 4
    return a


def make_params(box, rc=3.5, r0=2.5, sw_n=6, sw_m=12, stretch=True, cn_unlike_only=True, n_cv=2) -> Params:
    p = Params()
    for a in range(3):
        p.box[a] = float(box[a])
    p.rc, p.r0, p.sw_n, p.sw_m = float(rc), float(r0), int(sw_n), int(sw_m)
    p.stretch, p.cn_unlike_only, p.n_cv = int(bool(stretch)), int(bool(cn_unlike_only)), int(n_cv)
    return p


def params_from(mp, box) -> Params:
    """From a synth.MethodParams."""
    return make_params(box, mp.rc, mp.r0, mp.sw_n, mp.sw_m, True, mp.cn_unlike_only, mp.n_cv)


# ------------------------------------------------------------- neighbours
def pairs_brute(pos4, box, rc) -> np.ndarray:
    """Every unordered pair {i<j} with r^2 < rc^2 by the O(N^2) definition."""
    pos4 = _f32x4(pos4)
    b = np.ascontiguousarray(box, dtype=np.float64)
    n = pos4.shape[0]
    cap = max(16, n * 64)
    while True:
        out = np.empty((cap, 2), dtype=np.int64)
        np_ = _L().orc_pairs_brute(n, _ptr(pos4), _ptr(b), float(rc), _ptr(out), cap)
        if np_ >= 0:
            return out[:np_].copy()
        cap = -np_ - 1


def pairs_cells(pos4, box, rc, nthreads=0) -> np.ndarray:
    pos4 = _f32x4(pos4)
    b = np.ascontiguousarray(box, dtype=np.float64)
    n = pos4.shape[0]
    cap = max(16, n * 32)
    while True:
        out = np.empty((cap, 2), dtype=np.int64)
        np_ = _L().orc_pairs_cells(n, _ptr(pos4), _ptr(b), float(rc), _ptr(out), cap, int(nthreads))
        if np_ == -1:
            raise MemoryError("orc_pairs_cells failed")
        if np_ >= 0:
            return out[:np_].copy()
        cap = -np_ - 1


# ------------------------------------------------------------- pieces
def switch(p: Params, r):
    r = np.ascontiguousarray(r, dtype=np.float64).ravel()
    s, ds = np.empty_like(r), np.empty_like(r)
    _L().orc_switch(ctypes.byref(p), r.size, _ptr(r), _ptr(s), _ptr(ds))
    return s, ds


def ylm6(d):
    """Complex Y_6^m (m=-6..6) of direction d/|d| and dY/dd: ([n,13], [n,13,3])."""
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    n = d.shape[0]
    yr, yi = np.empty((n, 13)), np.empty((n, 13))
    gr, gi = np.empty((n, 13, 3)), np.empty((n, 13, 3))
    _L().orc_ylm(n, _ptr(d), _ptr(yr), _ptr(yi), _ptr(gr), _ptr(gi))
    return yr + 1j * yi, gr + 1j * gi


def cv(pos4, p: Params, nthreads=0):
    """(s[n_cv], cn[N], qbar6[N])."""
    pos4 = _f32x4(pos4)
    n = pos4.shape[0]
    s = np.zeros(2)
    cn, q6 = np.zeros(n), np.zeros(n)
    rc = _L().orc_cv(n, _ptr(pos4), ctypes.byref(p), _ptr(s), _ptr(cn), _ptr(q6), int(nthreads))
    if rc != 0:
        raise MemoryError("orc_cv failed")
    return s[: p.n_cv].copy(), cn, q6


def forces(pos4, p: Params, dVds, nthreads=0):
    """F = -sum_d dVds[d] * ds_d/dr  -> ([N,3] float64, s)."""
    pos4 = _f32x4(pos4)
    n = pos4.shape[0]
    dv = np.zeros(2)
    dv[: p.n_cv] = np.asarray(dVds, dtype=np.float64)[: p.n_cv]
    F = np.zeros((n, 3))
    s = np.zeros(2)
    rc = _L().orc_forces(n, _ptr(pos4), ctypes.byref(p), _ptr(dv), _ptr(F), _ptr(s), int(nthreads))
    if rc != 0:
        raise MemoryError("orc_forces failed")
    return F, s[: p.n_cv].copy()


class HillGrid:
    """Bicubic-Hermite bias grid: nodes [n0, n1, 4] = V, dV/ds0, dV/ds1, d2V/ds0ds1."""

    def __init__(self, n, lo, hi):
        self.n = (int(n[0]), int(n[1]))
        self.lo = (float(lo[0]), float(lo[1]))
        self.hi = (float(hi[0]), float(hi[1]))
        self.data = np.zeros((self.n[0], self.n[1], 4))

    def struct(self) -> Grid:
        g = Grid()
        g.n[0], g.n[1] = self.n
        g.lo[0], g.lo[1] = self.lo
        g.hi[0], g.hi[1] = self.hi
        g.data = self.data.ctypes.data
        return g

    def fold(self, centres, heights, sigma, nthreads=0):
        c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 2)
        w = np.ascontiguousarray(heights, dtype=np.float64)
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        g = self.struct()
        _L().orc_grid_fold(ctypes.byref(g), c.shape[0], _ptr(c), _ptr(w), _ptr(sg), int(nthreads))


def _grid_ref(grid):
    return None if grid is None else ctypes.byref(grid.struct())


def _period(period, ncv):
    if period is None:
        return None
    return np.ascontiguousarray(np.broadcast_to(np.asarray(period, dtype=np.float64), (ncv,)))


def bias(s, centres, heights, sigma, grid: HillGrid | None = None, period=None):
    """V(s) and dV/ds from hills (and grid).  period: None, or one period per
    CV (0 = not periodic; 2 pi for a torsion angle)."""
    s = np.ascontiguousarray(np.atleast_1d(s), dtype=np.float64)
    ncv = s.size
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, ncv)
    w = np.ascontiguousarray(heights, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    pr = _period(period, ncv)
    V = ctypes.c_double(0.0)
    dV = np.zeros(5)
    _L().orc_bias(ncv, _ptr(s), c.shape[0], _ptr(c), _ptr(w), _ptr(sg), _ptr(pr), _grid_ref(grid), ctypes.byref(V),
                  _ptr(dV))
    return V.value, dV[:ncv].copy()


def deposit_sequence(centres, sigma, w0, kbdt, grid: HillGrid | None = None, heights_prefix=None, period=None):
    """Well-tempered heights of hills deposited in order at the given centres."""
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    ncv = sg.size
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, ncv)
    K = c.shape[0]
    w = np.zeros(K)
    k0 = 0
    if heights_prefix is not None:
        k0 = len(heights_prefix)
        w[:k0] = heights_prefix
    pr = _period(period, ncv)
    _L().orc_deposit_sequence(ncv, K, k0, _ptr(c), _ptr(w), _ptr(sg), _ptr(pr), float(w0), float(kbdt),
                              _grid_ref(grid))
    return w


def step(pos4, p: Params, centres, heights, sigma, grid: HillGrid | None = None, nthreads=0):
    """One frame: neighbours, CVs, bias, forces -> dict(s, V, dV, F)."""
    pos4 = _f32x4(pos4)
    n = pos4.shape[0]
    ncv = p.n_cv
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, ncv)
    w = np.ascontiguousarray(heights, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    s, dV, F = np.zeros(2), np.zeros(2), np.zeros((n, 3))
    V = ctypes.c_double(0.0)
    rc = _L().orc_step(n, _ptr(pos4), ctypes.byref(p), c.shape[0], _ptr(c), _ptr(w), _ptr(sg), _grid_ref(grid),
                       _ptr(s), ctypes.byref(V), _ptr(dV), _ptr(F), int(nthreads))
    if rc != 0:
        raise MemoryError("orc_step failed")
    return {"s": s[:ncv].copy(), "V": V.value, "dV": dV[:ncv].copy(), "F": F}


def step_box(pos4, p: Params, centres, heights, sigma, lattice=True, nthreads=0):
    """One frame with the box derivative a barostat needs (Section "B4-B1
    phase transition in Large-scale systems": CN and the triaxial lattice
    parameters as CVs under NPT).  With lattice, the CVs are (s1 [, s2],
    L_x, L_y, L_z) and the hills D = n_cv + 3 dimensional.
    -> dict(s, V, dV, F, box_grad) with box_grad = dV/dL_a at fixed
    fractional coordinates (the explicit lattice term plus the bias virial
    over L_a)."""
    pos4 = _f32x4(pos4)
    n = pos4.shape[0]
    D = p.n_cv + (3 if lattice else 0)
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, D)
    w = np.ascontiguousarray(heights, dtype=np.float64)
    sg = np.ascontiguousarray(sigma, dtype=np.float64)
    assert sg.size == D
    s, dV, F, bg = np.zeros(5), np.zeros(5), np.zeros((n, 3)), np.zeros(3)
    V = ctypes.c_double(0.0)
    rc = _L().orc_step_box(n, _ptr(pos4), ctypes.byref(p), 1 if lattice else 0, c.shape[0], _ptr(c), _ptr(w),
                           _ptr(sg), _ptr(s), ctypes.byref(V), _ptr(dV), _ptr(F), _ptr(bg), int(nthreads))
    if rc != 0:
        raise MemoryError("orc_step_box failed")
    return {"s": s[:D].copy(), "V": V.value, "dV": dV[:D].copy(), "F": F, "box_grad": bg}


# ------------------------------------------------------------------ free energy
# Methods, after Eqs. 2-3: the bias fills the free-energy surface; the FES is
# recovered by reweighting the biased ensemble (Eq. 4: P_unbias(s) =
# <delta(s - s(R)) exp(beta V)> / <exp(beta V)>, Eq. 5: F = -(1/beta) log P).
# For a well-tempered bias the deposited bias itself estimates it: V(s) ->
# -(1 - 1/gamma) F(s) + const (the standard well-tempered limit; the paper
# names well-tempered MetaD but prints no formula, read here as that limit).

def fes_points(points, centres, heights, sigma, biasfactor, grid: HillGrid | None = None, period=None):
    """Sum-of-hills FES at each point: F = -(gamma / (gamma - 1)) V, shifted
    so that its minimum over the points is 0 (gamma = inf, plain
    metadynamics: F = -V)."""
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    V = np.array([bias(p, centres, heights, sigma, grid, period=period)[0] for p in pts])
    fac = 1.0 if np.isinf(biasfactor) else biasfactor / (biasfactor - 1.0)
    F = -fac * V
    return F - F.min()


def bin_index(s, lo, hi, n):
    """Bin of CV point s on the regular grid [lo, hi) with n bins per
    dimension (row-major, the first CV slowest); -1 when outside."""
    idx = 0
    for d in range(len(n)):
        h = (hi[d] - lo[d]) / n[d]
        if not (s[d] >= lo[d] and s[d] < hi[d]):
            return -1
        b = int(np.floor((s[d] - lo[d]) / h))
        if b >= n[d]:
            return -1
        idx = idx * n[d] + b
    return idx


def fes_reweight(samples, V, beta, lo, hi, n):
    """Eqs. 4-5 on a histogram: P_b = sum_{t in b} exp(beta V_t) / sum_t
    exp(beta V_t) over the samples inside the grid, F_b = -(1/beta) log P_b,
    shifted to minimum 0; empty bins are +inf.  Sums run in sample order,
    with exp(beta (V_t - max V)) for range."""
    S = np.atleast_2d(np.asarray(samples, dtype=np.float64))
    V = np.asarray(V, dtype=np.float64)
    nb = int(np.prod(n))
    vmax = V.max()
    acc = np.zeros(nb)
    tot = 0.0
    for t in range(S.shape[0]):
        b = bin_index(S[t], lo, hi, n)
        if b < 0:
            continue
        wt = np.exp(beta * (V[t] - vmax))
        acc[b] += wt
        tot += wt
    F = np.full(nb, np.inf)
    nz = acc > 0
    F[nz] = -np.log(acc[nz] / tot) / beta
    if nz.any():
        F[nz] -= F[nz].min()
    return F

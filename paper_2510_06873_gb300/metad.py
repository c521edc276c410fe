"""Thin Python binding of the C ABI in include/metad.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own; all work runs in the CUDA kernels of libmetad.so.
Device buffers are torch tensors (``tensor.data_ptr()``); host outputs are
numpy arrays.  If the library has not been built, importing this module
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmetad.so")

METAD_OK, METAD_ERR_INVALID, METAD_ERR_OOM, METAD_ERR_CUDA, METAD_ERR_CAPACITY, METAD_ERR_TIMEOUT, \
    METAD_ERR_STATE = range(7)
METAD_CV_COORDINATION, METAD_CV_TORSION, METAD_CV_NEAREST = range(3)
CV_KINDS = {"coordination": METAD_CV_COORDINATION, "torsion": METAD_CV_TORSION, "nearest": METAD_CV_NEAREST}


class metad_params(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("n_cv", ctypes.c_int32), ("box", ctypes.c_double * 3),
        ("rc", ctypes.c_double), ("r0", ctypes.c_double), ("sw_n", ctypes.c_int32), ("sw_m", ctypes.c_int32),
        ("stretch", ctypes.c_int32), ("cn_pairs", ctypes.c_int32), ("sigma", ctypes.c_double * 2),
        ("w0", ctypes.c_double), ("biasfactor", ctypes.c_double), ("temperature", ctypes.c_double),
        ("kB", ctypes.c_double), ("grid_on", ctypes.c_int32), ("grid_n", ctypes.c_int32 * 2),
        ("hill_capacity", ctypes.c_int32), ("grid_lo", ctypes.c_double * 2), ("grid_hi", ctypes.c_double * 2),
        ("precision", ctypes.c_int32), ("max_neighbors", ctypes.c_int32), ("device", ctypes.c_int32),
        ("step_graph", ctypes.c_int32), ("stream", ctypes.c_void_p), ("skin", ctypes.c_double),
        ("cv_kind", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("softmin_beta", ctypes.c_double),
        ("lattice_cvs", ctypes.c_int32), ("virial", ctypes.c_int32), ("sigma_lattice", ctypes.c_double * 3),
    ]


class MetadError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status}) {detail}".rstrip())


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "metad_params_default": (None, [ctypes.POINTER(metad_params)]),
    "metad_create": (ctypes.c_int, [ctypes.POINTER(metad_params), ctypes.POINTER(ctypes.c_void_p)]),
    "metad_destroy": (ctypes.c_int, [_P]),
    "metad_build_neighbors": (ctypes.c_int, [_P, _P]),
    "metad_cv_forward": (ctypes.c_int, [_P, _P, _P]),
    "metad_bias_eval": (ctypes.c_int, [_P, _P, _P, _P]),
    "metad_bias_forces": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_double]),
    "metad_deposit_hill": (ctypes.c_int, [_P, _P, _P]),
    "metad_set_cv_atoms": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "metad_set_box": (ctypes.c_int, [_P, _P]),
    "metad_box_gradient": (ctypes.c_int, [_P, _P]),
    "metad_deposit_hills": (ctypes.c_int, [_P, _P, ctypes.c_int32, _P]),
    "metad_load_hills": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "metad_get_hills": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "metad_fold_hills": (ctypes.c_int, [_P]),
    "metad_get_grid": (ctypes.c_int, [_P, _P]),
    "metad_export_neighbors": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "metad_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32]),
    "metad_read_results": (ctypes.c_int, [_P, _P, _P, _P]),
    "metad_sync": (ctypes.c_int, [_P]),
    "metad_stream": (ctypes.c_void_p, [_P]),
    "metad_hill_count": (ctypes.c_int32, [_P]),
    "metad_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "metad_last_error": (ctypes.c_char_p, [_P]),
    "metad_step_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "metad_profile_begin": (ctypes.c_int, [_P, ctypes.c_int32]),
    "metad_profile_end": (ctypes.c_int, [_P, _P, _P]),
    "metad_stage_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "metad_launch_count": (ctypes.c_int64, [_P]),
    "metad_neighbor_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "metad_rebuild_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "metad_bias_eval_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_int32,
                                               _P]),
    "metad_probe_recip": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_void_p]),
    "metad_probe_fp32_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_double)]),
    "metad_estimate_bytes": (ctypes.c_int, [ctypes.POINTER(metad_params), ctypes.POINTER(ctypes.c_int64)]),
    "metad_device_bytes": (ctypes.c_int64, [_P]),
    "metad_set_step_graph": (ctypes.c_int, [_P, ctypes.c_int32]),
    "metad_fes_grid": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "metad_cv_trajectory": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "metad_fes_reweight": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P, _P, _P]),
    "metad_batch_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "metad_batch_destroy": (ctypes.c_int, [_P]),
    "metad_batch_set_tile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "metad_batch_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P, _P]),
    "metad_batch_collect": (ctypes.c_int, [_P, _P]),
    "metad_batch_read": (ctypes.c_int, [_P, _P, _P]),
    "metad_batch_launch_count": (ctypes.c_int64, [_P]),
    "metad_batch_last_error": (ctypes.c_char_p, [_P]),
}
METAD_NUM_STAGES = 11
OPTIONAL = {}


def lib():
    """Load libmetad.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2510_06873_gb300.build.build() first "
                              "(the library has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in {**_SIGS, **OPTIONAL}.items():
            if not hasattr(L, name):
                if name in OPTIONAL:
                    continue
                raise ImportError(f"{LIB_PATH} does not export {name}")
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def status_string(s: int) -> str:
    try:
        return lib().metad_status_string(int(s)).decode()
    except ImportError:
        return str(s)


def _check(ctx, s, where):
    if s != METAD_OK:
        detail = ""
        if ctx:
            detail = lib().metad_last_error(ctx).decode()
        raise MetadError(s, where, detail)


def _dptr(t):
    """Device pointer of a torch tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _hptr(a):
    return None if a is None else a.ctypes.data


def metad_params_default() -> metad_params:
    p = metad_params()
    lib().metad_params_default(ctypes.byref(p))
    return p


def metad_create(p: metad_params):
    ctx = ctypes.c_void_p()
    s = lib().metad_create(ctypes.byref(p), ctypes.byref(ctx))
    _check(None, s, "metad_create")
    return ctx.value


def metad_destroy(ctx):
    lib().metad_destroy(ctx)


def metad_build_neighbors(ctx, pos):
    _check(ctx, lib().metad_build_neighbors(ctx, _dptr(pos)), "metad_build_neighbors")


def metad_cv_forward(ctx, n_cv=None, per_atom=None, want_host=True):
    """n_cv: the number of CVs D to return (n_cv, + 3 with lattice CVs)."""
    out = np.zeros(5) if want_host else None
    _check(ctx, lib().metad_cv_forward(ctx, _hptr(out), _dptr(per_atom)), "metad_cv_forward")
    return None if out is None else out[: (n_cv or 2)]


def metad_bias_eval(ctx, s=None, want_host=True):
    sh = None if s is None else np.ascontiguousarray(np.atleast_1d(s), dtype=np.float64)
    V = ctypes.c_double(0.0)
    dV = np.zeros(5)
    if want_host:
        _check(ctx, lib().metad_bias_eval(ctx, _hptr(sh), ctypes.byref(V), _hptr(dV)), "metad_bias_eval")
        return V.value, dV
    _check(ctx, lib().metad_bias_eval(ctx, _hptr(sh), None, None), "metad_bias_eval")
    return None


def metad_bias_forces(ctx, forces, accumulate=False, scale=1.0):
    _check(ctx, lib().metad_bias_forces(ctx, _dptr(forces), int(bool(accumulate)), float(scale)),
           "metad_bias_forces")


def metad_set_cv_atoms(ctx, atoms):
    a = np.ascontiguousarray(np.asarray(atoms).ravel(), dtype=np.int32)
    _check(ctx, lib().metad_set_cv_atoms(ctx, _hptr(a), int(a.size)), "metad_set_cv_atoms")


def metad_set_box(ctx, box):
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).ravel()[:3])
    _check(ctx, lib().metad_set_box(ctx, _hptr(b)), "metad_set_box")


def metad_box_gradient(ctx):
    out = np.zeros(3)
    _check(ctx, lib().metad_box_gradient(ctx, _hptr(out)), "metad_box_gradient")
    return out


def metad_deposit_hill(ctx, center=None, want_height=True):
    c = None if center is None else np.ascontiguousarray(np.atleast_1d(center), dtype=np.float64)
    h = ctypes.c_double(0.0)
    _check(ctx, lib().metad_deposit_hill(ctx, _hptr(c), ctypes.byref(h) if want_height else None),
           "metad_deposit_hill")
    return h.value if want_height else None


def metad_deposit_hills(ctx, centers, want_heights=True):
    c = np.ascontiguousarray(centers, dtype=np.float64)
    K = c.shape[0]
    w = np.zeros(K) if want_heights else None
    _check(ctx, lib().metad_deposit_hills(ctx, _hptr(c), K, _hptr(w)), "metad_deposit_hills")
    return w


def metad_load_hills(ctx, centers, heights):
    c = np.ascontiguousarray(centers, dtype=np.float64)
    w = np.ascontiguousarray(heights, dtype=np.float64)
    _check(ctx, lib().metad_load_hills(ctx, _hptr(c), _hptr(w), int(w.size)), "metad_load_hills")


def metad_get_hills(ctx, n_cv):
    K = ctypes.c_int32(0)
    _check(ctx, lib().metad_get_hills(ctx, None, None, 0, ctypes.byref(K)), "metad_get_hills")
    c = np.zeros((K.value, n_cv))
    w = np.zeros(K.value)
    _check(ctx, lib().metad_get_hills(ctx, _hptr(c), _hptr(w), K.value, ctypes.byref(K)), "metad_get_hills")
    return c, w


def metad_fold_hills(ctx):
    _check(ctx, lib().metad_fold_hills(ctx), "metad_fold_hills")


def metad_get_grid(ctx, shape):
    g = np.zeros((shape[0], shape[1], 4))
    _check(ctx, lib().metad_get_grid(ctx, _hptr(g)), "metad_get_grid")
    return g


def metad_export_neighbors(ctx):
    P = ctypes.c_int64(0)
    _check(ctx, lib().metad_export_neighbors(ctx, None, 0, ctypes.byref(P)), "metad_export_neighbors")
    out = np.zeros((P.value, 2), dtype=np.int64)
    _check(ctx, lib().metad_export_neighbors(ctx, _hptr(out), P.value, ctypes.byref(P)), "metad_export_neighbors")
    return out


def metad_step(ctx, pos, forces, accumulate=False, deposit=False):
    _check(ctx, lib().metad_step(ctx, _dptr(pos), _dptr(forces), int(bool(accumulate)), int(bool(deposit))),
           "metad_step")


def metad_step_host(ctx, pos_host, forces_host, accumulate=False, deposit=False):
    """pos_host float32 [N,4], forces_host float32 [N,3] (numpy, ideally pinned)."""
    cv = np.zeros(5)
    V = ctypes.c_double(0.0)
    _check(ctx, lib().metad_step_host(ctx, _hptr(pos_host), _hptr(forces_host), int(bool(accumulate)),
                                      int(bool(deposit)), _hptr(cv), ctypes.byref(V)), "metad_step_host")
    return cv, V.value


def metad_profile_begin(ctx, max_records):
    _check(ctx, lib().metad_profile_begin(ctx, int(max_records)), "metad_profile_begin")


def metad_profile_end(ctx):
    ms = np.zeros(METAD_NUM_STAGES)
    cnt = np.zeros(METAD_NUM_STAGES, dtype=np.int32)
    _check(ctx, lib().metad_profile_end(ctx, _hptr(ms), _hptr(cnt)), "metad_profile_end")
    return {metad_stage_name(k): (float(ms[k]), int(cnt[k])) for k in range(METAD_NUM_STAGES)}


def metad_stage_name(k) -> str:
    return lib().metad_stage_name(int(k)).decode()


def metad_neighbor_stats(ctx):
    e, mx = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(ctx, lib().metad_neighbor_stats(ctx, ctypes.byref(e), ctypes.byref(mx)), "metad_neighbor_stats")
    return int(e.value), int(mx.value)


def metad_rebuild_count(ctx) -> int:
    v = ctypes.c_int64(0)
    _check(ctx, lib().metad_rebuild_count(ctx, ctypes.byref(v)), "metad_rebuild_count")
    return int(v.value)


def metad_launch_count(ctx) -> int:
    return int(lib().metad_launch_count(ctx))


def metad_bias_eval_noalloc(s, centers, heights, sigma, out, device=None, stream=None):
    """s [n_cv], centers [K, n_cv], heights [K], out [>= 3]: float64 CUDA
    tensors, contiguous, on one device; sigma: host sequence of n_cv widths.
    device defaults to the tensors' device.  Asynchronous on `stream`;
    allocates nothing.  Tensors of the wrong type, shape or device raise
    MetadError(METAD_ERR_INVALID) before any device call (the kernel would
    otherwise read or write past the caller's buffers)."""
    import torch
    sg = np.ascontiguousarray(np.atleast_1d(sigma), dtype=np.float64)
    n_cv = int(sg.size)
    where = "metad_bias_eval_noalloc"
    tensors = {"s": s, "centers": centers, "heights": heights, "out": out}
    for name, t in tensors.items():
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise MetadError(METAD_ERR_INVALID, where, f"{name} must be a contiguous float64 CUDA tensor")
    devs = {t.device.index for t in tensors.values()}
    if len(devs) != 1:
        raise MetadError(METAD_ERR_INVALID, where, "tensors on different devices")
    dev_index = devs.pop()
    if device is None:
        device = dev_index
    elif int(device) != dev_index:
        raise MetadError(METAD_ERR_INVALID, where, f"tensors on cuda:{dev_index}, device {device} named")
    K = int(heights.shape[0]) if heights.dim() == 1 else -1
    if K < 0 or centers.shape != (K, n_cv) and not (K == 0 and centers.numel() == 0):
        raise MetadError(METAD_ERR_INVALID, where, f"centers must be [K, n_cv] = [{K}, {n_cv}]")
    if s.numel() < n_cv or out.numel() < 3:
        raise MetadError(METAD_ERR_INVALID, where, "s needs n_cv entries and out at least 3")
    _check(None, lib().metad_bias_eval_noalloc(_dptr(s), n_cv, _dptr(centers), _dptr(heights), K, _hptr(sg),
                                               _dptr(out), int(device), stream), where)


def metad_probe_recip(v, out, which, stream=None):
    """out = f(v) on the device for a test of the kernels' FP32 reciprocals:
    which 0 / 2 the kernels' 1/sqrt / 1/v, 1 / 3 CUDA's correctly rounded ones.
    v, out: contiguous float32 CUDA tensors of the same size."""
    import torch
    for t in (v, out):
        if not (isinstance(t, torch.Tensor) and t.dtype == torch.float32 and t.is_contiguous() and t.is_cuda):
            raise MetadError(METAD_ERR_INVALID, "metad_probe_recip", "float32 contiguous CUDA tensors")
    if v.numel() != out.numel():
        raise MetadError(METAD_ERR_INVALID, "metad_probe_recip", "sizes differ")
    _check(None, lib().metad_probe_recip(ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         int(v.numel()), int(which), stream), "metad_probe_recip")


def metad_probe_fp32_peak(device=0, iters=16384, repeats=20):
    """Measured FP32 multiply-add throughput of `device` in TFLOP/s (the
    roofline denominator of the ALU-bound kernels).  Synchronises."""
    v = ctypes.c_double(0.0)
    _check(None, lib().metad_probe_fp32_peak(int(device), int(iters), int(repeats), ctypes.byref(v)),
           "metad_probe_fp32_peak")
    return v.value


def metad_read_results(ctx):
    cv, dV = np.zeros(5), np.zeros(5)
    V = ctypes.c_double(0.0)
    _check(ctx, lib().metad_read_results(ctx, _hptr(cv), ctypes.byref(V), _hptr(dV)), "metad_read_results")
    return cv, V.value, dV


def metad_sync(ctx):
    _check(ctx, lib().metad_sync(ctx), "metad_sync")


def metad_stream(ctx) -> int:
    return int(lib().metad_stream(ctx) or 0)


def metad_hill_count(ctx) -> int:
    return int(lib().metad_hill_count(ctx))


# --------------------------------------------------------------------- helper
def params_for(n_atoms, box, n_cv=2, sigma=(0.05, 0.02), rc=3.5, r0=2.5, sw_n=6, sw_m=12, cn_unlike=True,
               w0=1.0, biasfactor=10.0, temperature=300.0, kB=0.0083144626, grid=None, hill_capacity=65536,
               fp64=False, max_neighbors=64, device=0, stream=None, skin=1.0, step_graph=False,
               cv_kind="coordination", softmin_beta=0.0, lattice_cvs=False, virial=False,
               sigma_lattice=(0.1, 0.1, 0.1)) -> metad_params:
    """metad_params from keyword values; grid = (n, lo, hi) or None; cv_kind
    "coordination", "torsion" or "nearest" (or the METAD_CV_* value)."""
    p = metad_params_default()
    p.n_atoms = int(n_atoms)
    p.n_cv = int(n_cv)
    for a in range(3):
        p.box[a] = float(box[a])
    p.rc, p.r0, p.sw_n, p.sw_m = float(rc), float(r0), int(sw_n), int(sw_m)
    p.cn_pairs = 1 if cn_unlike else 0
    sig = list(sigma) + [1.0] * (2 - len(sigma))
    p.sigma[0], p.sigma[1] = float(sig[0]), float(sig[1])
    p.w0, p.biasfactor, p.temperature, p.kB = float(w0), float(biasfactor), float(temperature), float(kB)
    if grid is not None:
        gn, lo, hi = grid
        p.grid_on = 1
        p.grid_n[0], p.grid_n[1] = int(gn[0]), int(gn[1])
        p.grid_lo[0], p.grid_lo[1] = float(lo[0]), float(lo[1])
        p.grid_hi[0], p.grid_hi[1] = float(hi[0]), float(hi[1])
    p.hill_capacity = int(hill_capacity)
    p.precision = 1 if fp64 else 0
    p.max_neighbors = int(max_neighbors)
    p.device = int(device)
    p.stream = stream
    p.skin = float(skin)
    p.step_graph = 1 if step_graph else 0
    p.cv_kind = CV_KINDS[cv_kind] if isinstance(cv_kind, str) else int(cv_kind)
    p.softmin_beta = float(softmin_beta)
    p.lattice_cvs = 1 if lattice_cvs else 0
    p.virial = 1 if virial else 0
    for a in range(3):
        p.sigma_lattice[a] = float(sigma_lattice[a])
    return p


class Metad:
    """One context: owns the C handle, forwards to the metad_* calls."""

    def __init__(self, params: metad_params):
        self.params = params
        self.n = params.n_atoms
        # CVs the hills see (and every CV vector in and out): the per-atom
        # CVs, then the box lengths with lattice CVs
        self.n_cv = params.n_cv + (3 if params.lattice_cvs else 0)
        self.ctx = metad_create(params)

    def close(self):
        if getattr(self, "ctx", None):
            metad_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def build_neighbors(self, pos):
        metad_build_neighbors(self.ctx, pos)

    def cv_forward(self, per_atom=None, want_host=True):
        out = metad_cv_forward(self.ctx, self.n_cv, per_atom, want_host)
        return out

    def bias_eval(self, s=None, want_host=True):
        r = metad_bias_eval(self.ctx, s, want_host)
        if r is None:
            return None
        return r[0], r[1][: self.n_cv]

    def bias_forces(self, forces, accumulate=False, scale=1.0):
        metad_bias_forces(self.ctx, forces, accumulate, scale)

    def set_cv_atoms(self, atoms):
        metad_set_cv_atoms(self.ctx, atoms)

    def set_box(self, box):
        metad_set_box(self.ctx, box)

    def box_gradient(self):
        return metad_box_gradient(self.ctx)

    def deposit_hill(self, center=None, want_height=True):
        return metad_deposit_hill(self.ctx, center, want_height)

    def deposit_hills(self, centers, want_heights=True):
        return metad_deposit_hills(self.ctx, centers, want_heights)

    def load_hills(self, centers, heights):
        metad_load_hills(self.ctx, centers, heights)

    def get_hills(self):
        return metad_get_hills(self.ctx, self.n_cv)

    def fold_hills(self):
        metad_fold_hills(self.ctx)

    def get_grid(self):
        return metad_get_grid(self.ctx, (self.params.grid_n[0], self.params.grid_n[1]))

    def export_neighbors(self):
        return metad_export_neighbors(self.ctx)

    def step(self, pos, forces, accumulate=False, deposit=False):
        metad_step(self.ctx, pos, forces, accumulate, deposit)

    def read_results(self):
        cv, V, dV = metad_read_results(self.ctx)
        return cv[: self.n_cv], V, dV[: self.n_cv]

    def sync(self):
        metad_sync(self.ctx)

    def step_host(self, pos_host, forces_host, accumulate=False, deposit=False):
        cv, V = metad_step_host(self.ctx, pos_host, forces_host, accumulate, deposit)
        return cv[: self.n_cv], V

    def profile_begin(self, max_records):
        metad_profile_begin(self.ctx, max_records)

    def profile_end(self):
        return metad_profile_end(self.ctx)

    def neighbor_stats(self):
        return metad_neighbor_stats(self.ctx)

    @property
    def rebuild_count(self) -> int:
        return metad_rebuild_count(self.ctx)

    @property
    def launch_count(self) -> int:
        return metad_launch_count(self.ctx)

    @property
    def stream(self) -> int:
        return metad_stream(self.ctx)

    @property
    def hill_count(self) -> int:
        return metad_hill_count(self.ctx)

    @property
    def device_bytes(self) -> int:
        return metad_device_bytes(self.ctx)

    def set_step_graph(self, on: bool):
        metad_set_step_graph(self.ctx, on)

    def cv_trajectory(self, frames):
        return metad_cv_trajectory(self.ctx, frames, self.params.n_cv)

    def fes_grid(self, lo, hi, n):
        return metad_fes_grid(self.ctx, lo, hi, n)

    def fes_reweight(self, samples, V, lo, hi, n):
        return metad_fes_reweight(self.ctx, samples, V, lo, hi, n)


def metad_estimate_bytes(p: metad_params) -> int:
    out = ctypes.c_int64(0)
    _check(None, lib().metad_estimate_bytes(ctypes.byref(p), ctypes.byref(out)), "metad_estimate_bytes")
    return int(out.value)


def metad_device_bytes(ctx) -> int:
    return int(lib().metad_device_bytes(ctx))


def metad_set_step_graph(ctx, on: bool):
    _check(ctx, lib().metad_set_step_graph(ctx, 1 if on else 0), "metad_set_step_graph")


def _grid_args(lo, hi, n):
    lo_a = np.zeros(2)
    hi_a = np.zeros(2)
    n_a = np.ones(2, dtype=np.int32)
    k = len(n)
    lo_a[:k], hi_a[:k], n_a[:k] = lo, hi, n
    return lo_a, hi_a, n_a


def metad_fes_grid(ctx, lo, hi, n):
    """F at the bin centres of the grid, shape tuple(n)."""
    lo_a, hi_a, n_a = _grid_args(lo, hi, n)
    F = np.zeros(int(np.prod(n)))
    _check(ctx, lib().metad_fes_grid(ctx, _hptr(lo_a), _hptr(hi_a), _hptr(n_a), _hptr(F)), "metad_fes_grid")
    return F.reshape(tuple(n))


def metad_cv_trajectory(ctx, frames, n_cv):
    """CVs of every frame of a device tensor [T, N, 4]; returns [T, n_cv]."""
    T = int(frames.shape[0])
    out = np.zeros((T, 2))
    _check(ctx, lib().metad_cv_trajectory(ctx, _dptr(frames), T, _hptr(out)), "metad_cv_trajectory")
    return out[:, :n_cv]


def metad_fes_reweight(ctx, samples, V, lo, hi, n):
    """Reweighted F on the grid's bins, shape tuple(n) (+inf where empty)."""
    lo_a, hi_a, n_a = _grid_args(lo, hi, n)
    S = np.ascontiguousarray(samples, dtype=np.float64)
    Va = np.ascontiguousarray(V, dtype=np.float64)
    F = np.zeros(int(np.prod(n)))
    _check(ctx, lib().metad_fes_reweight(ctx, _hptr(S), _hptr(Va), len(Va), _hptr(lo_a), _hptr(hi_a), _hptr(n_a),
                                         _hptr(F)), "metad_fes_reweight")
    return F.reshape(tuple(n))


# ------------------------------------------------------------------ batches

def _bcheck(batch, s, where):
    if s != METAD_OK:
        detail = lib().metad_batch_last_error(batch).decode() if batch else ""
        raise MetadError(s, where, detail)


def metad_batch_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    out = ctypes.c_void_p()
    _bcheck(None, lib().metad_batch_create(arr, len(ctxs), ctypes.byref(out)), "metad_batch_create")
    return out


def metad_batch_destroy(batch):
    lib().metad_batch_destroy(batch)


def metad_batch_set_tile(batch, blocks_per_system):
    _bcheck(batch, lib().metad_batch_set_tile(batch, int(blocks_per_system)), "metad_batch_set_tile")


def metad_batch_step(batch, pos_list, force_list, accumulate=False, deposit=None, active=None):
    """pos_list / force_list: one tensor (or None when inactive) per system."""
    n = len(pos_list)
    pos = (ctypes.c_void_p * n)(*[_dptr(t) for t in pos_list])
    frc = (ctypes.c_void_p * n)(*[_dptr(t) for t in force_list])
    dep_a = None if deposit is None else np.ascontiguousarray(np.asarray(deposit, dtype=np.int32))
    act_a = None if active is None else np.ascontiguousarray(np.asarray(active, dtype=np.int32))
    _bcheck(batch, lib().metad_batch_step(batch, pos, frc, 1 if accumulate else 0, _hptr(dep_a), _hptr(act_a)),
            "metad_batch_step")


def metad_batch_collect(batch, out_host):
    """out_host: float64 numpy array [n, 4] (page-locked for an asynchronous copy)."""
    _bcheck(batch, lib().metad_batch_collect(batch, _hptr(out_host)), "metad_batch_collect")


def metad_batch_read(batch, n):
    cv = np.zeros((n, 2), dtype=np.float64)
    V = np.zeros(n, dtype=np.float64)
    _bcheck(batch, lib().metad_batch_read(batch, _hptr(cv), _hptr(V)), "metad_batch_read")
    return cv, V


def metad_batch_launch_count(batch) -> int:
    return lib().metad_batch_launch_count(batch)


class Batch:
    """Many contexts stepped together, one launch per stage (metad_batch_*).

    The contexts stay owned by the caller and must outlive the batch."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        self.n = len(self.contexts)
        self.batch = metad_batch_create([c.ctx for c in self.contexts])

    def close(self):
        if getattr(self, "batch", None):
            metad_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile(self, blocks_per_system):
        metad_batch_set_tile(self.batch, blocks_per_system)

    def step(self, pos_list, force_list, accumulate=False, deposit=None, active=None):
        metad_batch_step(self.batch, pos_list, force_list, accumulate, deposit, active)

    def collect(self, out_host):
        metad_batch_collect(self.batch, out_host)

    def read(self):
        """(cv [n, 2], V [n]) of the last batched step; synchronises."""
        return metad_batch_read(self.batch, self.n)

    @property
    def launch_count(self) -> int:
        return metad_batch_launch_count(self.batch)

"""The bias as a torch.autograd.Function: gradients against finite differences.

* small system, FP64 pair mode: central differences of the GPU's own V with
  full recompute (h = 2^-13 A);
* the recompute path: a backward after the context has run another frame;
* 1M atoms, FP32 pairs, the full grid + 20,000-hill bias: 64 random atoms,
  central differences h = 2^-13 A (about 1e-4 A) computed in FP64 by local
  recompute in the oracle -- only atoms within 2 rc of the moved atom change
  their CVs, and those depend on atoms within 4 rc, so a non-periodic
  cluster of radius 4 rc around it gives the exact change of s -- turned into
  dV by the chain rule with the oracle's dV/ds.  Atoms with a pair within 2h
  of rc are redrawn (the switch has a kink there).
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import kbdt, setup_hills

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H = 2.0 ** -13
RC = 3.5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06873_gb300 import build
    build.build()
    d = torch.device("cuda:0")
    torch.cuda.set_stream(torch.cuda.Stream(d))
    return d


def _ctx(dev, n, box, mp, fp64=False, grid=None, cap=65536):
    from paper_2510_06873_gb300 import autograd, metad
    p = metad.params_for(n, box, n_cv=mp.n_cv, sigma=mp.sigma, fp64=fp64, grid=grid, hill_capacity=cap,
                         stream=torch.cuda.current_stream(dev).cuda_stream)
    return autograd.BiasContext(p)


def test_fp64_gradient_matches_central_differences(dev):
    from paper_2510_06873_gb300 import autograd
    system = synth.wurtzite_system(3000, cfg=98)
    mp = synth.MethodParams(n_cv=2)
    c, s0 = setup_hills(system, mp, 400, cfg=98)
    ctx = _ctx(dev, system.n, system.box, mp, fp64=True)
    ctx.deposit_hills(c)
    frame = synth.perturbed_frame(system, 1)
    pos = torch.from_numpy(frame).to(dev).requires_grad_(True)
    V = autograd.bias(pos, ctx)
    V.backward()
    g = pos.grad.cpu().numpy().astype(np.float64)
    assert np.all(g[:, 3] == 0.0)
    rng = np.random.default_rng(0)
    worst = 0.0
    for k in rng.choice(system.n, 8, replace=False):
        for a in range(3):
            fp, fm = frame.copy(), frame.copy()
            fp[k, a] = np.float32(frame[k, a] + np.float32(H))
            fm[k, a] = np.float32(frame[k, a] - np.float32(H))
            h2 = float(fp[k, a]) - float(fm[k, a])
            Vp = float(autograd.bias(torch.from_numpy(fp).to(dev), ctx))
            Vm = float(autograd.bias(torch.from_numpy(fm).to(dev), ctx))
            worst = max(worst, abs((Vp - Vm) / h2 - g[k, a]))
    assert worst <= 1e-6 * np.abs(g[:, :3]).max()
    # the oracle's gradient of the same frame: dV/dr = -F(dV/ds), with the
    # oracle's own CVs and bias gradient (FP64 pairs on both sides, the
    # gradient stored in float32)
    p = oracle.params_from(mp, system.box)
    w = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    ref = oracle.step(frame, p, c, w, mp.sigma)
    g_ref = -ref["F"]
    nrm = np.linalg.norm(g[:, :3] - g_ref) / np.linalg.norm(g_ref)
    per = np.max(np.linalg.norm(g[:, :3] - g_ref, axis=1)) / np.max(np.linalg.norm(g_ref, axis=1))
    assert nrm <= 2e-7 and per <= 2e-7, (nrm, per)
    ctx.close()


def test_backward_recomputes_after_context_moves_on(dev):
    from paper_2510_06873_gb300 import autograd
    system = synth.wurtzite_system(5000, cfg=99)
    mp = synth.MethodParams(n_cv=2)
    c, _ = setup_hills(system, mp, 300, cfg=99)
    ctx = _ctx(dev, system.n, system.box, mp)
    ctx.deposit_hills(c)
    fa, fb = synth.perturbed_frame(system, 0), synth.perturbed_frame(system, 1)
    pa = torch.from_numpy(fa).to(dev).requires_grad_(True)
    Va = autograd.bias(pa, ctx)
    Va.backward()
    ga = pa.grad.clone()
    pa.grad = None
    Va2 = autograd.bias(pa, ctx)
    Vb = autograd.bias(torch.from_numpy(fb).to(dev), ctx)  # the context moves on
    Va2.backward()                                          # must recompute frame a
    assert torch.equal(pa.grad, ga)
    assert float(Va2) == float(Va) and float(Vb) != float(Va)
    ctx.close()


def _cluster_delta_s(frame, box, p_big, m, axis, h):
    """FP64 change of (sum CN, sum qbar6) over atoms within 2 rc of atom m when
    m moves from -h to +h along axis: exact local recompute in a cluster."""
    x = frame[:, :3].astype(np.float64)
    d = x - x[m]
    d -= box * np.round(d / box)
    r = np.linalg.norm(d, axis=1)
    sel = np.nonzero(r < 4 * RC + 0.5)[0]
    near = r[sel] < 2 * RC + 0.5
    centre = 50.0
    out = []
    for sgn in (+1, -1):
        cl = np.zeros((sel.size, 4), np.float32)
        cl[:, :3] = (d[sel] + centre).astype(np.float32)
        cl[:, 3] = frame[sel, 3]
        im = int(np.nonzero(sel == m)[0][0])
        cl[im, :3] = np.float32(centre)
        cl[im, axis] = np.float32(centre + sgn * h)
        _, cn, q6 = oracle.cv(cl, p_big)
        out.append((cn[near].sum(), q6[near].sum()))
    return np.array(out[0]) - np.array(out[1])


@pytest.mark.slow
def test_config3_autograd_against_local_finite_differences(dev):
    from paper_2510_06873_gb300 import autograd
    system = synth.config3_system()
    mp = synth.method_params(3)
    cfgp = synth.CONFIG_PARAMS[3]
    K1, K2 = cfgp["hills_folded"], cfgp["hills"]
    cen, s_ref = setup_hills(system, mp, K1 + K2, cfg=3)
    sig = np.asarray(mp.sigma)
    lo, hi = s_ref - 16 * sig, s_ref + 16 * sig
    w1 = oracle.deposit_sequence(cen[:K1], mp.sigma, mp.w0, kbdt(mp))
    G = oracle.HillGrid(cfgp["grid_n"], lo, hi)
    G.fold(cen[:K1], w1, mp.sigma)
    w2 = oracle.deposit_sequence(cen[K1:], mp.sigma, mp.w0, kbdt(mp), grid=G)
    ctx = _ctx(dev, system.n, system.box, mp, grid=(cfgp["grid_n"], lo, hi))
    ctx.deposit_hills(cen[:K1], want_heights=False)
    ctx.fold_hills()
    ctx.deposit_hills(cen[K1:], want_heights=False)
    frame = synth.perturbed_frame(system, 0)
    pos = torch.from_numpy(frame).to(dev).requires_grad_(True)
    V = autograd.bias(pos, ctx)
    V.backward()
    g = pos.grad.cpu().numpy().astype(np.float64)[:, :3]
    # oracle CVs and bias gradient of the full frame
    p = oracle.params_from(mp, system.box)
    s0, _, _ = oracle.cv(frame, p)
    _, dV = oracle.bias(s0, cen[K1:], w2, mp.sigma, grid=G)
    p_big = oracle.params_from(mp, [100.0, 100.0, 100.0])
    pairs = oracle.pairs_cells(frame, system.box, RC)
    x = frame[:, :3].astype(np.float64)
    rng = np.random.default_rng(64)
    gmax = np.abs(g).max()
    checked = 0
    for m in rng.permutation(system.n):
        if checked == 64:
            break
        nb = np.concatenate([pairs[pairs[:, 0] == m, 1], pairs[pairs[:, 1] == m, 0]])
        dd = x[nb] - x[m]
        dd -= system.box * np.round(dd / system.box)
        rr = np.linalg.norm(dd, axis=1)
        if np.any(np.abs(rr - RC) < 4 * H):
            continue  # a pair near the switch kink at rc: redraw
        fd = np.zeros(3)
        for a in range(3):
            ds = _cluster_delta_s(frame, system.box, p_big, m, a, H) / system.n
            fd[a] = (dV[0] * ds[0] + dV[1] * ds[1]) / (2 * H)
        err = np.linalg.norm(g[m] - fd)
        assert err <= 1e-4 * np.linalg.norm(fd) + 1e-6 * gmax, (m, g[m], fd)
        checked += 1
    assert checked == 64
    ctx.close()

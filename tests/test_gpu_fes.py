"""Free-energy passes (metad_fes_grid, metad_fes_reweight) against the FP64
oracle: the well-tempered sum-of-hills estimate on a grid (with and without
the bias grid) and Eqs. 4-5 reweighting of biased samples."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import kbdt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06873_gb300 import build
    build.build()
    d = torch.device("cuda:0")
    torch.cuda.set_stream(torch.cuda.Stream(d))
    return d


def _ctx(dev, n_cv, grid=None):
    from paper_2510_06873_gb300 import metad
    sig = (0.05, 0.02)[:n_cv]
    p = metad.params_for(1000, [23.2, 23.2, 23.2], n_cv=n_cv, sigma=sig, grid=grid,
                         stream=torch.cuda.current_stream(dev).cuda_stream)
    return metad.Metad(p)


def centres_of(lo, hi, n):
    axes = [lo[d] + (np.arange(n[d]) + 0.5) * ((hi[d] - lo[d]) / n[d]) for d in range(len(n))]
    if len(n) == 1:
        return axes[0][:, None]
    return np.array([[a, b] for a in axes[0] for b in axes[1]])


@pytest.mark.parametrize("n_cv", [1, 2])
def test_sum_of_hills_fes_matches_oracle(dev, n_cv):
    mp = synth.MethodParams(n_cv=n_cv, sigma=(0.05, 0.02)[:n_cv])
    g = np.random.default_rng(40 + n_cv)
    sig = np.asarray(mp.sigma)
    ctr = np.array([2.0, 0.3])[:n_cv]
    c = ctr + g.uniform(-8, 8, size=(700, n_cv)) * sig
    ctx = _ctx(dev, n_cv)
    w = ctx.deposit_hills(c)
    w_ref = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    assert np.allclose(w, w_ref, rtol=1e-12, atol=0)
    lo, hi = ctr - 10 * sig, ctr + 10 * sig
    n = (37, 23)[:n_cv]
    F = ctx.fes_grid(lo, hi, n).ravel()
    ref = oracle.fes_points(centres_of(lo, hi, n), c, w_ref, mp.sigma, mp.biasfactor)
    assert np.abs(F - ref).max() <= 1e-10 * np.abs(ref).max()
    assert F.min() == 0.0


def test_fes_includes_the_bias_grid(dev):
    mp = synth.MethodParams(n_cv=2)
    sig = np.asarray(mp.sigma)
    ctr = np.array([2.0, 0.3])
    g = np.random.default_rng(47)
    c = ctr + g.uniform(-8, 8, size=(900, 2)) * sig
    lo_g, hi_g = ctr - 16 * sig, ctr + 16 * sig
    ctx = _ctx(dev, 2, grid=((60, 60), lo_g, hi_g))
    w1 = ctx.deposit_hills(c[:600])
    ctx.fold_hills()
    w2 = ctx.deposit_hills(c[600:])
    # the oracle's own heights: deposit, fold, deposit on top of the grid
    w1_ref = oracle.deposit_sequence(c[:600], mp.sigma, mp.w0, kbdt(mp))
    G = oracle.HillGrid((60, 60), lo_g, hi_g)
    G.fold(c[:600], w1_ref, mp.sigma)
    w2_ref = oracle.deposit_sequence(c[600:], mp.sigma, mp.w0, kbdt(mp), grid=G)
    assert np.allclose(w1, w1_ref, rtol=1e-12, atol=0) and np.allclose(w2, w2_ref, rtol=1e-11, atol=0)
    lo, hi, n = ctr - 9 * sig, ctr + 9 * sig, (31, 29)
    F = ctx.fes_grid(lo, hi, n).ravel()
    ref = oracle.fes_points(centres_of(lo, hi, n), c[600:], w2_ref, mp.sigma, mp.biasfactor, grid=G)
    assert np.abs(F - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("n_cv", [1, 2])
def test_reweighted_fes_matches_oracle(dev, n_cv):
    mp = synth.MethodParams(n_cv=n_cv, sigma=(0.05, 0.02)[:n_cv])
    g = np.random.default_rng(50 + n_cv)
    T = 20000
    S = np.column_stack([g.normal(2.0, 0.08, T), g.normal(0.3, 0.03, T)])[:, :n_cv]
    V = g.uniform(0.0, 15.0, T)
    lo, hi, n = (1.8, 0.22)[:n_cv], (2.2, 0.38)[:n_cv], (20, 16)[:n_cv]
    ctx = _ctx(dev, n_cv)
    F = ctx.fes_reweight(S, V, lo, hi, n).ravel()
    beta = 1.0 / (mp.kB * mp.temperature)
    ref = oracle.fes_reweight(S, V, beta, lo, hi, n)
    assert np.array_equal(np.isinf(F), np.isinf(ref))
    fin = ~np.isinf(ref)
    assert fin.sum() > 10
    assert np.allclose(F[fin], ref[fin], rtol=1e-11, atol=1e-11)


def test_reweight_edge_cases(dev):
    ctx = _ctx(dev, 1)
    # every sample outside the grid: every bin empty
    F = ctx.fes_reweight(np.array([[5.0], [6.0]]), np.array([1.0, 2.0]), (0.0,), (1.0,), (4,)).ravel()
    assert np.all(np.isinf(F))
    # one sample: its bin is 0, the rest empty
    F = ctx.fes_reweight(np.array([[0.3]]), np.array([1.0]), (0.0,), (1.0,), (4,)).ravel()
    assert F[1] == 0.0 and np.isinf(F[[0, 2, 3]]).all()
    from paper_2510_06873_gb300 import metad
    with pytest.raises(metad.MetadError):
        ctx.fes_reweight(np.array([[0.3]]), np.array([1.0]), (1.0,), (0.0,), (4,))

"""The allocation-free bias entry point against the context's bias_eval.

metad_bias_eval_noalloc serves callers that cannot allocate device memory
where they need the bias (an MD step pipelined on its own stream, where a
cudaMalloc could synchronise the device; a fixed memory budget; no library
context allowed).  It must give the same V and dV/ds as metad_bias_eval on
the same hills, call after call, while its scratch is shared between calls.
This file is collected last so that a failure here never hides another test.
"""
import numpy as np
import pytest

import synth

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


@pytest.mark.parametrize("n_cv,K", [(2, 5000), (2, 131072), (1, 777)])
def test_noalloc_matches_context_bias_twice(dev, n_cv, K):
    from paper_2510_06873_gb300 import metad
    sigma = (0.05, 0.02)[:n_cv]
    s_ref = np.array([2.7, 0.23])[:n_cv]
    centres = synth.hill_centres(97, K, s_ref, sigma, K)
    heights = synth.rng(97, K, 5).uniform(0.2, 1.0, K)
    stream = torch.cuda.current_stream(dev)
    # reference: the context path
    p = metad.params_for(10, [20.0, 20.0, 20.0], n_cv=n_cv, sigma=sigma, hill_capacity=K + 8,
                         stream=stream.cuda_stream)
    ctx = metad.Metad(p)
    ctx.load_hills(centres, heights)
    c_dev = torch.from_numpy(np.ascontiguousarray(centres)).to(dev)
    w_dev = torch.from_numpy(heights).to(dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    g = synth.rng(97, K, 6)
    for call in range(2):
        s = s_ref + g.normal(size=n_cv) * np.asarray(sigma)
        V_ref, dV_ref = ctx.bias_eval(s)
        s_dev = torch.from_numpy(s).to(dev)
        metad.metad_bias_eval_noalloc(s_dev, c_dev, w_dev, sigma, out, device=0, stream=stream.cuda_stream)
        got = out.cpu().numpy()
        assert abs(got[0] - V_ref) <= 1e-12 * max(abs(V_ref), 1.0), (call, got[0], V_ref)
        for d in range(n_cv):
            assert abs(got[1 + d] - dV_ref[d]) <= 1e-12 * max(abs(dV_ref[d]), 1.0 / sigma[d]), (call, d)
        if n_cv == 1:
            assert got[2] == 0.0, call
    ctx.close()


def test_noalloc_without_hills_writes_zero(dev):
    """K = 0 (the one-block path): V and dV/ds are 0, on two calls after a
    call that left non-zero partials in the shared scratch."""
    from paper_2510_06873_gb300 import metad
    st = torch.cuda.current_stream(dev).cuda_stream
    out = torch.full((3,), 7.0, dtype=torch.float64, device=dev)
    s = torch.tensor([2.7, 0.23], dtype=torch.float64, device=dev)
    c1 = torch.tensor([[2.7, 0.23]], dtype=torch.float64, device=dev)
    w1 = torch.tensor([0.5], dtype=torch.float64, device=dev)
    metad.metad_bias_eval_noalloc(s, c1, w1, (0.05, 0.02), out, stream=st)
    assert out.cpu().numpy()[0] == 0.5
    for n_cv in (2, 1):
        c0 = torch.zeros((0, n_cv), dtype=torch.float64, device=dev)
        w0 = torch.zeros(0, dtype=torch.float64, device=dev)
        out.fill_(7.0)
        metad.metad_bias_eval_noalloc(s, c0, w0, (0.05, 0.02)[:n_cv], out, stream=st)
        assert np.array_equal(out.cpu().numpy(), np.zeros(3)), n_cv


def test_noalloc_rejects_bad_tensors(dev):
    """The binding refuses tensors the kernel would overrun or misread."""
    from paper_2510_06873_gb300 import metad
    st = torch.cuda.current_stream(dev).cuda_stream
    s = torch.zeros(2, dtype=torch.float64, device=dev)
    c = torch.zeros((4, 2), dtype=torch.float64, device=dev)
    w = torch.zeros(4, dtype=torch.float64, device=dev)
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    bad = [(s.float(), c, w, out), (s, c[:, :1].clone(), w, out), (s, c, w, out[:2]), (s, c.t(), w, out),
           (s, c, w.cpu(), out)]
    for args in bad:
        with pytest.raises(metad.MetadError) as e:
            metad.metad_bias_eval_noalloc(args[0], args[1], args[2], (0.05, 0.02), args[3], stream=st)
        assert e.value.status == metad.METAD_ERR_INVALID


def test_noalloc_rejects_too_many_hills(dev):
    from paper_2510_06873_gb300 import metad
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    s = torch.zeros(2, dtype=torch.float64, device=dev)
    c = torch.zeros((131073, 2), dtype=torch.float64, device=dev)
    w = torch.zeros(131073, dtype=torch.float64, device=dev)
    with pytest.raises(metad.MetadError) as e:
        metad.metad_bias_eval_noalloc(s, c, w, (0.05, 0.02), out, stream=torch.cuda.current_stream(dev).cuda_stream)
    assert e.value.status == metad.METAD_ERR_CAPACITY

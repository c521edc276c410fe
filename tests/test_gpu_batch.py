"""Batched form (many systems, one launch per stage) through the C ABI.

The systems follow the batched workload: wurtzite/liquid systems with atom
counts log-uniform over a range, each with its own density factor in
[0.9, 1.1] and its own well-tempered hill history.  With the default tile a
batched step must give every system the same bits as stepping its context
alone; every system must match the FP64 oracle within the tolerances of
parity_util; a tile setting changes no result (the CV sums have a grid of
their own).
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_bias, check_cv, check_forces, kbdt, setup_hills

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


def _metad():
    from paper_2510_06873_gb300 import metad
    return metad


def layout(count, n_hi, k_hi):
    n, k, dens = synth.batch_layout(4, n_systems=count, n_hi=n_hi, k_hi=k_hi)
    systems = [synth.wurtzite_system(int(n[s]), cfg=4, sys=s, density_scale=float(dens[s])) for s in range(count)]
    return systems, [int(x) for x in k]


def make_ctx(dev, system, mp, cap=None, stream=None):
    metad = _metad()
    st = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
    p = metad.params_for(system.n, system.box, n_cv=2, sigma=mp.sigma, stream=st,
                         hill_capacity=cap if cap is not None else 65536)
    return metad.Metad(p)


@pytest.fixture(scope="module")
def small_batch(dev):
    mp = synth.method_params(4)
    systems, ks = layout(6, 2e4, 600)
    hills = [setup_hills(s, mp, k, cfg=4)[0] for s, k in zip(systems, ks)]
    return mp, systems, hills


def frames_for(systems, f, dev):
    return [torch.from_numpy(synth.perturbed_frame(s, f)).to(dev) for s in systems]


def test_batched_step_is_bitwise_the_single_step(dev, small_batch):
    metad = _metad()
    mp, systems, hills = small_batch
    A = [make_ctx(dev, s, mp) for s in systems]
    B = [make_ctx(dev, s, mp) for s in systems]
    for a, b, c in zip(A, B, hills):
        ha = a.deposit_hills(c)
        hb = b.deposit_hills(c)
        assert np.array_equal(ha, hb)
    batch = metad.Batch(A)
    FA = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    FB = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    for f in range(3):
        pos = frames_for(systems, f, dev)
        dep = [1 if (f == 1 and k % 2 == 1) else 0 for k in range(len(systems))]
        batch.step(pos, FA, deposit=dep)
        cvA, VA = batch.read()
        for k, b in enumerate(B):
            b.step(pos[k], FB[k], deposit=bool(dep[k]))
            cvB, VB, _ = b.read_results()
            assert np.array_equal(cvA[k], cvB), (f, k, cvA[k], cvB)
            assert VA[k] == VB, (f, k)
            assert torch.equal(FA[k], FB[k]), (f, k)
    for a, b in zip(A, B):
        assert a.hill_count == b.hill_count
        ca, wa = a.get_hills()
        cb, wb = b.get_hills()
        assert np.array_equal(ca, cb) and np.array_equal(wa, wb)
    # one launch per stage for all systems: the gather, six rebuild
    # kernels, two CV kernels (the second with the CV sums), the bias,
    # adjoint, pair and gather force kernels (plus one deposit and one
    # collect where they ran)
    assert batch.launch_count == 3 * 13 + 1 + 3
    batch.close()


def test_batched_systems_match_the_oracle(dev, small_batch):
    metad = _metad()
    mp, systems, hills = small_batch
    ctxs = [make_ctx(dev, s, mp) for s in systems]
    w_gpu = [c.deposit_hills(h) for c, h in zip(ctxs, hills)]
    batch = metad.Batch(ctxs)
    F = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    f = 7
    pos = frames_for(systems, f, dev)
    batch.step(pos, F)
    cv, V = batch.read()
    for k, s in enumerate(systems):
        w_ref = oracle.deposit_sequence(hills[k], mp.sigma, mp.w0, kbdt(mp))
        assert np.allclose(w_gpu[k], w_ref, rtol=1e-12, atol=0)
        ref = oracle.step(synth.perturbed_frame(s, f), oracle.params_from(mp, s.box), hills[k], w_ref, mp.sigma)
        check_cv(cv[k], ref["s"])
        _, _, dV = ctxs[k].read_results()
        check_bias(V[k], dV, ref["V"], ref["dV"], mp)
        check_forces(F[k].cpu().numpy().astype(np.float64), ref["F"])
    batch.close()


def test_tile_setting_changes_no_result(dev, small_batch):
    metad = _metad()
    mp, systems, hills = small_batch
    A = [make_ctx(dev, s, mp) for s in systems]
    B = [make_ctx(dev, s, mp) for s in systems]
    for a, b, c in zip(A, B, hills):
        a.deposit_hills(c, want_heights=False)
        b.deposit_hills(c, want_heights=False)
    ba, bb = metad.Batch(A), metad.Batch(B)
    bb.set_tile(3)
    FA = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    FB = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    pos = frames_for(systems, 2, dev)
    ba.step(pos, FA)
    bb.step(pos, FB)
    cva, Va = ba.read()
    cvb, Vb = bb.read()
    assert np.array_equal(cva, cvb) and np.array_equal(Va, Vb)
    for fa, fb in zip(FA, FB):
        assert torch.equal(fa, fb)
    ba.close()
    bb.close()


def test_autotuner_picks_a_candidate(dev, small_batch):
    metad = _metad()
    from paper_2510_06873_gb300 import tune
    mp, systems, hills = small_batch
    ctxs = [make_ctx(dev, s, mp) for s in systems]
    for c, h in zip(ctxs, hills):
        c.deposit_hills(h, want_heights=False)
    batch = metad.Batch(ctxs)
    F = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    pos = frames_for(systems, 0, dev)
    r = tune.tune_batch(batch, pos, F, torch.cuda.current_stream(dev), candidates=(0, 64, 8), steps=2)
    assert r["tile"] in (0, 64, 8) and set(r["ms_per_step"]) == {0, 64, 8}
    assert all(v > 0 for v in r["ms_per_step"].values())
    assert all(c.hill_count == len(h) for c, h in zip(ctxs, hills))
    batch.close()


def test_inactive_systems_are_untouched(dev, small_batch):
    metad = _metad()
    mp, systems, hills = small_batch
    A = [make_ctx(dev, s, mp) for s in systems]
    B = [make_ctx(dev, s, mp) for s in systems]
    for a, b, c in zip(A, B, hills):
        a.deposit_hills(c, want_heights=False)
        b.deposit_hills(c, want_heights=False)
    batch = metad.Batch(A)
    FA = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    FB = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    act = [1, 0, 1, 0, 0, 1]
    for f in range(2):
        pos = frames_for(systems, f, dev)
        batch.step([p if a else None for p, a in zip(pos, act)], [x if a else None for x, a in zip(FA, act)],
                   deposit=[1] * len(systems), active=act)
        cvA, VA = batch.read()
        for k, b in enumerate(B):
            if not act[k]:
                continue
            b.step(pos[k], FB[k], deposit=True)
            cvB, VB, _ = b.read_results()
            assert np.array_equal(cvA[k], cvB) and VA[k] == VB and torch.equal(FA[k], FB[k])
    for k in range(len(systems)):
        want = len(hills[k]) + (2 if act[k] else 0)
        assert A[k].hill_count == want
        assert float(FA[k].abs().sum()) == 0.0 or act[k]
    batch.close()


def test_batch_errors(dev, small_batch):
    metad = _metad()
    mp, systems, hills = small_batch
    a = make_ctx(dev, systems[0], mp)
    other = torch.cuda.Stream(dev)
    b = make_ctx(dev, systems[1], mp, stream=other.cuda_stream)
    with pytest.raises(metad.MetadError) as e:
        metad.Batch([a, b])
    assert e.value.status == metad.METAD_ERR_INVALID
    batch = metad.Batch([a])
    with pytest.raises(metad.MetadError) as e:
        batch.read()
    assert e.value.status == metad.METAD_ERR_STATE
    full = make_ctx(dev, systems[0], mp, cap=1)
    full.deposit_hills(hills[0][:1], want_heights=False)
    fb = metad.Batch([full])
    pos = frames_for(systems[:1], 0, dev)
    F = [torch.zeros((systems[0].n, 3), dtype=torch.float32, device=dev)]
    with pytest.raises(metad.MetadError) as e:
        fb.step(pos, F, deposit=[1])
    assert e.value.status == metad.METAD_ERR_CAPACITY
    fb.step(pos, F, deposit=[0])  # a refused step leaves the batch usable
    fb.read()
    batch.close()
    fb.close()


@pytest.mark.slow
def test_full_batched_workload(dev):
    """All 64 systems (1k-200k atoms, 100-10,000 hills): two batched steps
    bitwise equal to the single steps; sampled systems against the oracle."""
    metad = _metad()
    mp = synth.method_params(4)
    cfgp = synth.CONFIG_PARAMS[4]
    systems, ks = layout(cfgp["systems"], 2e5, 1e4)
    print("batched workload atoms", sum(s.n for s in systems), "hills", sum(ks))
    hills = [setup_hills(s, mp, k, cfg=4)[0] for s, k in zip(systems, ks)]
    A = [make_ctx(dev, s, mp) for s in systems]
    B = [make_ctx(dev, s, mp) for s in systems]
    for a, b, c in zip(A, B, hills):
        a.deposit_hills(c, want_heights=False)
        b.deposit_hills(c, want_heights=False)
    batch = metad.Batch(A)
    FA = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    FB = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    for f in range(2):
        pos = frames_for(systems, f, dev)
        batch.step(pos, FA)
        cvA, VA = batch.read()
        for k, b in enumerate(B):
            b.step(pos[k], FB[k])
        torch.cuda.synchronize(dev)
        for k, b in enumerate(B):
            cvB, VB, _ = b.read_results()
            assert np.array_equal(cvA[k], cvB) and VA[k] == VB and torch.equal(FA[k], FB[k]), k
    order = np.argsort([s.n for s in systems])
    for k in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        s = systems[k]
        w_ref = oracle.deposit_sequence(hills[k], mp.sigma, mp.w0, kbdt(mp))
        ref = oracle.step(synth.perturbed_frame(s, 1), oracle.params_from(mp, s.box), hills[k], w_ref, mp.sigma)
        check_cv(cvA[k], ref["s"])
        _, _, dV = A[k].read_results()
        check_bias(VA[k], dV, ref["V"], ref["dV"], mp)
        check_forces(FA[k].cpu().numpy().astype(np.float64), ref["F"])
        # the neighbour set the batched step used, bit for bit
        pairs = A[k].export_neighbors()
        assert np.array_equal(pairs, oracle.pairs_cells(synth.perturbed_frame(s, 1), s.box, 3.5)), k
    batch.close()


def test_batched_fp64_single_cv_systems(dev):
    """The FP64, coordination-number-only configuration batched: bitwise the
    single steps, and the oracle's CVs and forces."""
    metad = _metad()
    mp = synth.method_params(1)
    systems = [synth.rsa_liquid_system(n, 0.08, 1.8, cfg=96, sys=k) for k, n in enumerate((500, 1000, 1700))]
    A, B = [], []
    for s in systems:
        for lst in (A, B):
            p = metad.params_for(s.n, s.box, n_cv=1, sigma=mp.sigma, fp64=True,
                                 stream=torch.cuda.current_stream(dev).cuda_stream)
            lst.append(metad.Metad(p))
    hills = [setup_hills(s, mp, 150, cfg=96)[0] for s in systems]
    for a, b, c in zip(A, B, hills):
        a.deposit_hills(c, want_heights=False)
        b.deposit_hills(c, want_heights=False)
    batch = metad.Batch(A)
    FA = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    FB = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
    pos = frames_for(systems, 3, dev)
    batch.step(pos, FA, deposit=[0, 1, 0])
    cvA, VA = batch.read()
    for k, (s, b) in enumerate(zip(systems, B)):
        b.step(pos[k], FB[k], deposit=(k == 1))
        cvB, VB, _ = b.read_results()
        assert cvA[k][0] == cvB[0] and cvA[k][1] == 0.0 and VA[k] == VB
        assert torch.equal(FA[k], FB[k])
        w_ref = oracle.deposit_sequence(hills[k], mp.sigma, mp.w0, kbdt(mp))
        ref = oracle.step(synth.perturbed_frame(s, 3), oracle.params_from(mp, s.box), hills[k], w_ref, mp.sigma)
        check_cv(cvA[k][:1], ref["s"])
        check_forces(FA[k].cpu().numpy().astype(np.float64), ref["F"])
    assert A[1].hill_count == 151
    batch.close()

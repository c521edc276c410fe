"""Torsion and nearest-distance CV families on the GPU against the FP64 oracle.

Workloads: seeded 22-atom chain molecules with two backbone torsions sharing
three atoms (Phi / Psi of the alanine-dipeptide runs), hills uniform on the
torus with sigma 0.35 rad; and a slab + water system whose CV is the
distance from one surface oxygen to its nearest hydrogen (the rutile runs),
exact and as a soft minimum.  Tolerances as every parity test (relative
1e-5 against FP64 with floors); angles get the floor 1 rad.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import geometric as og
from parity_util import check_forces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TWO_PI = 2.0 * math.pi
TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06873_gb300 import build
    build.build()
    d = torch.device("cuda:0")
    torch.cuda.set_stream(torch.cuda.Stream(d))
    return d


def _stream(dev):
    return torch.cuda.current_stream(dev)


def peptide_ctx(dev, biasfactor=math.inf, hill_capacity=20000, step_graph=False, fp64=False):
    from paper_2510_06873_gb300 import metad
    p = metad.params_for(synth.PEPTIDE_ATOMS, synth.peptide_box(), n_cv=2, sigma=(0.35, 0.35), w0=1.2,
                         biasfactor=biasfactor, cv_kind="torsion", hill_capacity=hill_capacity,
                         stream=_stream(dev).cuda_stream, step_graph=step_graph, fp64=fp64)
    ctx = metad.Metad(p)
    ctx.set_cv_atoms(synth.PEPTIDE_TORSIONS)
    return ctx


def surface_ctx(dev, sw, beta=0.0, hill_capacity=4000):
    from paper_2510_06873_gb300 import metad
    p = metad.params_for(sw.n, sw.box, n_cv=1, sigma=(0.1,), w0=1.0, biasfactor=10.0, cv_kind="nearest",
                         softmin_beta=beta, hill_capacity=hill_capacity, stream=_stream(dev).cuda_stream)
    ctx = metad.Metad(p)
    ctx.set_cv_atoms(sw.cv_atoms())
    return ctx


def kbdt_of(biasfactor):
    return synth.KB_KJMOL * 300.0 * (biasfactor - 1.0)


def check_angle(s, ref):
    for a, b in zip(np.atleast_1d(s), np.atleast_1d(ref)):
        assert abs(math.remainder(a - b, TWO_PI)) <= TOL * max(abs(b), 1.0), (s, ref)


def check_bias(V, dV, V_ref, dV_ref, w0, sigma):
    assert abs(V - V_ref) <= TOL * max(abs(V_ref), w0), (V, V_ref)
    for d in range(len(dV_ref)):
        assert abs(dV[d] - dV_ref[d]) <= TOL * max(abs(dV_ref[d]), w0 / sigma[d]), (dV, dV_ref)


def run_step(ctx, frame, dev, accumulate=False, F0=None, deposit=False):
    pos = torch.from_numpy(frame).to(dev)
    F = torch.zeros((frame.shape[0], 3), dtype=torch.float32, device=dev) if F0 is None else \
        torch.from_numpy(F0.copy()).to(dev)
    ctx.step(pos, F, accumulate=accumulate, deposit=deposit)
    cv, V, dV = ctx.read_results()
    return np.array(cv), V, np.array(dV), F.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("biasfactor,fp64", [(math.inf, False), (10.0, False), (10.0, True)])
def test_torsions_match_oracle(dev, biasfactor, fp64):
    """FP32 angle arithmetic (precision 0) and FP64 (precision 1)."""
    sig = (0.35, 0.35)
    c = synth.torus_centres(0, 3000)
    w = oracle.deposit_sequence(c, sig, 1.2, kbdt_of(biasfactor), period=[TWO_PI] * 2)
    if math.isinf(biasfactor):
        assert np.all(w == 1.2)
    ctx = peptide_ctx(dev, biasfactor, fp64=fp64)
    ctx.load_hills(c, w)
    box = synth.peptide_box()
    for f in range(12):
        fr = synth.peptide_frame(f)
        cv, V, dV, F = run_step(ctx, fr, dev)
        ref = og.step(fr, box, "torsion", synth.PEPTIDE_TORSIONS, 2, c, w, sig, period=[TWO_PI] * 2)
        check_angle(cv, ref["s"])
        check_bias(V, dV, ref["V"], ref["dV"], 1.2, sig)
        check_forces(F, ref["F"])
        assert np.all(F[[k for k in range(22) if k not in synth.PEPTIDE_TORSIONS[:8]]] == 0.0)
    ctx.close()


def test_torsion_deposits_wrap_across_the_seam(dev):
    """Deposit at each step's CVs; heights come from the periodic bias of all
    earlier hills, including those across the -pi/pi seam."""
    sig = (0.35, 0.35)
    ctx = peptide_ctx(dev, 10.0)
    box = synth.peptide_box()
    cvs = []
    for f in range(40):
        fr = synth.peptide_frame(100 + f)
        cv, _, _, _ = run_step(ctx, fr, dev, deposit=True)
        cvs.append(cv)
    c_gpu, w_gpu = ctx.get_hills()
    for f in range(40):
        ref = og.cvs(synth.peptide_frame(100 + f), box, "torsion", synth.PEPTIDE_TORSIONS, 2)
        check_angle(c_gpu[f], [ref[0][0], ref[1][0]])
        assert np.array_equal(c_gpu[f], cvs[f])
    w_ref = oracle.deposit_sequence(c_gpu, sig, 1.0 * 1.2, kbdt_of(10.0), period=[TWO_PI] * 2)
    assert np.abs(w_gpu - w_ref).max() <= TOL * 1.2
    assert w_gpu.min() < 1.2  # some hills saw earlier ones
    ctx.close()


@pytest.mark.parametrize("beta", [0.0, 8.0])
def test_nearest_distance_matches_oracle(dev, beta):
    sw = synth.SurfaceWater()
    sp = synth.SMALL_PARAMS["surface_water"]
    c = synth.interval_centres(synth.SURFACE_CFG, 0, 800, sp["cv_lo"], sp["cv_hi"])
    w = oracle.deposit_sequence(c, (0.1,), 1.0, kbdt_of(10.0))
    ctx = surface_ctx(dev, sw, beta)
    ctx.load_hills(c, w)
    atoms = sw.cv_atoms()
    for f in range(10):
        fr = sw.frame(f)
        cv, V, dV, F = run_step(ctx, fr, dev)
        ref = og.step(fr, sw.box, "min_dist", atoms, 1, c, w, (0.1,), beta=beta)
        assert abs(cv[0] - ref["s"][0]) <= TOL * abs(ref["s"][0])
        check_bias(V, dV, ref["V"], ref["dV"], 1.0, (0.1,))
        check_forces(F, ref["F"])
        moved = np.flatnonzero(np.any(F != 0.0, axis=1))
        if beta == 0.0:
            # only the reference and the nearest hydrogen move, and that
            # hydrogen is the oracle's (an FP64 decision on both sides)
            assert len(moved) == 2 and sw.ref in moved
            assert set(moved) == set(np.flatnonzero(np.any(ref["F"] != 0.0, axis=1)))
    ctx.close()


def test_accumulate_and_scale(dev):
    from paper_2510_06873_gb300 import metad
    ctx = peptide_ctx(dev)
    c = synth.torus_centres(1, 500)
    ctx.load_hills(c, np.full(500, 1.2))
    fr = synth.peptide_frame(7)
    base = np.random.default_rng(0).normal(size=(22, 3)).astype(np.float32)
    _, _, _, F1 = run_step(ctx, fr, dev)
    _, _, _, F2 = run_step(ctx, fr, dev, accumulate=True, F0=base)
    assert np.array_equal(F2.astype(np.float32), (base + F1.astype(np.float32)))
    pos = torch.from_numpy(fr).to(dev)
    F = torch.zeros((22, 3), dtype=torch.float32, device=dev)
    ctx.build_neighbors(pos)
    ctx.cv_forward()
    ctx.bias_eval()
    metad.metad_bias_forces(ctx.ctx, F, False, -2.0)
    assert np.array_equal(F.cpu().numpy(), (-2.0 * F1).astype(np.float32))
    ctx.close()


def test_degenerate_and_box_crossing_torsions(dev):
    box = synth.peptide_box()
    ctx = peptide_ctx(dev)
    ctx.load_hills(np.array([[0.1, 0.2]]), np.array([1.2]))
    fr = synth.peptide_frame(3)
    # the first torsion's four atoms collinear: angle 0, no force from it
    line = fr.copy()
    a, b, c_, d = synth.PEPTIDE_TORSIONS[:4]
    for k, at in enumerate((a, b, c_, d)):
        line[at, :3] = np.float32(5.0 + 1.5 * k)
    cv, _, _, F = run_step(ctx, line, dev)
    ref = og.step(line, box, "torsion", synth.PEPTIDE_TORSIONS, 2, np.array([[0.1, 0.2]]), np.array([1.2]),
                  (0.35, 0.35), period=[TWO_PI] * 2)
    assert cv[0] == 0.0 and ref["s"][0] == 0.0
    check_forces(F, ref["F"])
    # the molecule shifted so its bonds cross every face of the box
    shifted = fr.copy()
    shifted[:, :3] = synth.wrap_to_box(fr[:, :3].astype(np.float64) + (box - fr[b, :3]), box)
    cv2, _, _, F2 = run_step(ctx, shifted, dev)
    ref2 = og.step(shifted, box, "torsion", synth.PEPTIDE_TORSIONS, 2, np.array([[0.1, 0.2]]), np.array([1.2]),
                   (0.35, 0.35), period=[TWO_PI] * 2)
    check_angle(cv2, ref2["s"])
    check_angle(cv2, og.cvs(fr, box, "torsion", synth.PEPTIDE_TORSIONS, 2)[0][0])
    check_forces(F2, ref2["F"])
    ctx.close()


def test_batched_walkers_equal_single_steps(dev):
    """64 torsion walkers (own frames and hills) in one launch per stage give
    the bits of stepping each alone, deposits included."""
    from paper_2510_06873_gb300 import metad
    n = 64
    ctxs = [peptide_ctx(dev, 10.0, hill_capacity=4000) for _ in range(n)]
    solo = [peptide_ctx(dev, 10.0, hill_capacity=4000) for _ in range(n)]
    for k in range(n):
        c = synth.torus_centres(10 + k, 50 + 37 * k)
        w = np.full(len(c), 1.2)
        ctxs[k].load_hills(c, w)
        solo[k].load_hills(c, w)
    batch = metad.Batch(ctxs)
    pos = [torch.from_numpy(synth.peptide_frame(1000 + k)).to(dev) for k in range(n)]
    Fb = [torch.zeros((22, 3), dtype=torch.float32, device=dev) for _ in range(n)]
    Fs = [torch.zeros((22, 3), dtype=torch.float32, device=dev) for _ in range(n)]
    for step in range(3):
        dep = np.array([(k + step) % 3 == 0 for k in range(n)], dtype=np.int32)
        batch.step(pos, Fb, deposit=dep)
        cvb, Vb = batch.read()
        for k in range(n):
            solo[k].step(pos[k], Fs[k], deposit=bool(dep[k]))
            cv, V, _ = solo[k].read_results()
            assert np.array_equal(cvb[k], cv) and Vb[k] == V
            assert torch.equal(Fb[k], Fs[k])
    for k in range(n):
        assert all(np.array_equal(a, b) for a, b in zip(ctxs[k].get_hills(), solo[k].get_hills()))
    assert batch.launch_count == 3 * 1 + 3  # one fused launch per step, one collect per read
    batch.close()
    for c in ctxs + solo:
        c.close()


def test_batched_nearest_distance_against_oracle(dev):
    from paper_2510_06873_gb300 import metad
    systems = [synth.SurfaceWater(cells=(3 + k % 2, 3, 3), sys=k) for k in range(6)]
    ctxs = [surface_ctx(dev, sw, beta=(0.0 if k % 2 else 5.0)) for k, sw in enumerate(systems)]
    c = synth.interval_centres(synth.SURFACE_CFG, 1, 300, 0.9, 3.6)
    w = oracle.deposit_sequence(c, (0.1,), 1.0, kbdt_of(10.0))
    for x in ctxs:
        x.load_hills(c, w)
    batch = metad.Batch(ctxs)
    frames = [sw.frame(5) for sw in systems]
    pos = [torch.from_numpy(f).to(dev) for f in frames]
    F = [torch.zeros((sw.n, 3), dtype=torch.float32, device=dev) for sw in systems]
    batch.step(pos, F)
    cv, V = batch.read()
    for k, sw in enumerate(systems):
        ref = og.step(frames[k], sw.box, "min_dist", sw.cv_atoms(), 1, c, w, (0.1,), beta=(0.0 if k % 2 else 5.0))
        assert abs(cv[k, 0] - ref["s"][0]) <= TOL * ref["s"][0]
        assert abs(V[k] - ref["V"]) <= TOL * max(ref["V"], 1.0)
        check_forces(F[k].cpu().numpy().astype(np.float64), ref["F"])
    batch.close()
    for x in ctxs:
        x.close()


def test_trajectory_fes_and_graph_replay(dev):
    box = synth.peptide_box()
    frames = np.stack([synth.peptide_frame(200 + t) for t in range(16)])
    ctx = peptide_ctx(dev)
    cv = ctx.cv_trajectory(torch.from_numpy(frames).to(dev))
    for t in range(16):
        ref = [r[0] for r in og.cvs(frames[t], box, "torsion", synth.PEPTIDE_TORSIONS, 2)]
        check_angle(cv[t], ref)
    # sum-of-hills FES on the torus (plain metadynamics: F = -V)
    c = synth.torus_centres(3, 400)
    w = np.full(400, 1.2)
    ctx.load_hills(c, w)
    lo, hi, n = np.array([-math.pi, -math.pi]), np.array([math.pi, math.pi]), (24, 24)
    Fes = ctx.fes_grid(lo, hi, n).ravel()
    ax = [lo[d] + (np.arange(n[d]) + 0.5) * ((hi[d] - lo[d]) / n[d]) for d in range(2)]
    pts = np.array([[a, b] for a in ax[0] for b in ax[1]])
    ref = oracle.fes_points(pts, c, w, (0.35, 0.35), math.inf, period=[TWO_PI] * 2)
    assert np.abs(Fes - ref).max() <= 1e-10 * np.abs(ref).max()
    ctx.close()
    # graph replay gives the direct step's bits
    g = peptide_ctx(dev, step_graph=True)
    d = peptide_ctx(dev)
    for x in (g, d):
        x.load_hills(c, w)
    for f in range(5):
        a = run_step(g, synth.peptide_frame(f), dev)
        b = run_step(d, synth.peptide_frame(f), dev)
        assert all(np.array_equal(x, y) for x, y in zip(a, b))
    g.close()
    d.close()


def test_large_system_takes_the_three_kernel_path(dev):
    """Above the fused-step size the step runs as CV pass, hill kernel and
    force pass; it agrees with the oracle and with the separate calls."""
    from paper_2510_06873_gb300 import metad
    n = 40000
    g = np.random.default_rng(8)
    box = np.array([80.0, 80.0, 80.0])
    fr = np.zeros((n, 4), dtype=np.float32)
    fr[:, :3] = g.uniform(0, 80, (n, 3))
    atoms = np.concatenate([[7], g.choice(np.arange(100, n), 3000, replace=False)]).astype(np.int32)
    p = metad.params_for(n, box, n_cv=1, sigma=(0.1,), cv_kind="nearest", softmin_beta=3.0,
                         stream=_stream(dev).cuda_stream)
    ctx = metad.Metad(p)
    ctx.set_cv_atoms(atoms)
    s0 = og.cvs(fr, box, "min_dist", atoms, 1, 3.0)[0][0]
    c = (s0 + np.linspace(-1.0, 1.0, 60))[:, None]  # hills around the CV
    w = oracle.deposit_sequence(c, (0.1,), 1.0, kbdt_of(10.0))
    ctx.load_hills(c, w)
    l0 = ctx.launch_count
    cv, V, dV, F = run_step(ctx, fr, dev)
    assert ctx.launch_count - l0 == 3
    ref = og.step(fr, box, "min_dist", atoms, 1, c, w, (0.1,), beta=3.0)
    assert abs(cv[0] - ref["s"][0]) <= TOL * ref["s"][0]
    check_bias(V, dV, ref["V"], ref["dV"], 1.0, (0.1,))
    check_forces(F, ref["F"])
    ctx.close()


def test_small_family_errors(dev):
    from paper_2510_06873_gb300 import metad
    p = metad.params_for(22, synth.peptide_box(), n_cv=2, sigma=(0.35, 0.35), cv_kind="torsion",
                         stream=_stream(dev).cuda_stream)
    ctx = metad.Metad(p)
    pos = torch.from_numpy(synth.peptide_frame(0)).to(dev)
    ctx.build_neighbors(pos)
    with pytest.raises(metad.MetadError) as e:
        ctx.cv_forward()
    assert e.value.status == metad.METAD_ERR_STATE
    ctx.close()
    for bad in ([0, 1, 2], [0, 1, 2, 3, 4, 5, 6, 99], [0, 1, 1, 2, 3, 4, 5, 6]):
        ctx = metad.Metad(p)
        with pytest.raises(metad.MetadError) as e:
            ctx.set_cv_atoms(bad)
        assert e.value.status == metad.METAD_ERR_INVALID
        ctx.close()
    ctx = peptide_ctx(dev)
    with pytest.raises(metad.MetadError) as e:
        ctx.export_neighbors()
    assert e.value.status == metad.METAD_ERR_INVALID
    ctx.close()
    sw = synth.SurfaceWater()
    q = metad.params_for(sw.n, sw.box, n_cv=1, sigma=(0.1,), cv_kind="nearest", stream=_stream(dev).cuda_stream)
    for bad in ([sw.ref], [sw.ref, sw.ref, 1], [sw.ref, 5, 5]):
        ctx = metad.Metad(q)
        with pytest.raises(metad.MetadError) as e:
            ctx.set_cv_atoms(bad)
        assert e.value.status == metad.METAD_ERR_INVALID
        ctx.close()
    # a non-finite position is reported, not hidden
    ctx = peptide_ctx(dev)
    fr = synth.peptide_frame(0)
    fr[synth.PEPTIDE_TORSIONS[0], 0] = np.nan
    with pytest.raises(metad.MetadError):
        run_step(ctx, fr, dev)
    ctx.close()

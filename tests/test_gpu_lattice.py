"""Lattice-parameter CVs and the box gradient (NPT) on the GPU against the
FP64 oracle.

The GaN NPT runs bias the coordination number together with the triaxial
lattice parameters.  Frames follow a triaxial NPT run: each box length is
scaled by 1 + e_a per frame (positions with it, plus thermal noise); the
context gets the box by metad_set_box before each step.  Checked: the CVs
(s1 [, s2], L_x, L_y, L_z), the D-dimensional bias and its gradient, the
forces, dV/dL at fixed fractional coordinates (lattice term plus the bias
virial), deposits, neighbour sets after box changes (cells shrinking and
capped), batched steps bit for bit, and the error paths.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_forces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
SIG_L = (0.1, 0.1, 0.1)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06873_gb300 import build
    build.build()
    d = torch.device("cuda:0")
    torch.cuda.set_stream(torch.cuda.Stream(d))
    return d


@pytest.fixture(scope="module")
def system():
    return synth.wurtzite_system(8000, cfg=8)


def kbdt():
    return synth.KB_KJMOL * 300.0 * 9.0


def make_ctx(dev, system, n_cv, lattice=True, virial=False, hills=None):
    from paper_2510_06873_gb300 import metad
    p = metad.params_for(system.n, system.box, n_cv=n_cv, sigma=(0.05, 0.02)[:n_cv], lattice_cvs=lattice,
                         virial=virial, sigma_lattice=SIG_L, stream=torch.cuda.current_stream(dev).cuda_stream)
    ctx = metad.Metad(p)
    if hills is not None:
        ctx.load_hills(*hills)
    return ctx


def lattice_hills(system, n_cv, count=400, lattice=True):
    p = oracle.make_params(system.box, n_cv=n_cv)
    s0 = oracle.cv(system.base, p)[0][:n_cv]
    sig = np.array(list((0.05, 0.02)[:n_cv]) + (list(SIG_L) if lattice else []))
    ref = np.concatenate([s0, system.box]) if lattice else s0
    c = synth.hill_centres(8, 0, ref, sig, count, half_width_sigmas=4.0)
    w = oracle.deposit_sequence(c, sig, 1.0, kbdt())
    return c, w, sig


def run(ctx, frame, dev, box=None, deposit=False):
    if box is not None:
        ctx.set_box(box)
    pos = torch.from_numpy(frame).to(dev)
    F = torch.zeros((frame.shape[0], 3), dtype=torch.float32, device=dev)
    ctx.step(pos, F, deposit=deposit)
    cv, V, dV = ctx.read_results()
    return np.array(cv), V, np.array(dV), F.cpu().numpy().astype(np.float64)


def check_box_grad(bg, ref, sig_floor):
    scale = max(np.abs(ref).max(), 1.0 / sig_floor)
    assert np.abs(np.asarray(bg) - ref).max() <= TOL * scale, (bg, ref)


@pytest.mark.parametrize("n_cv", [1, 2])
def test_npt_sequence_matches_oracle(dev, system, n_cv):
    c, w, sig = lattice_hills(system, n_cv)
    ctx = make_ctx(dev, system, n_cv, hills=(c, w))
    for f in range(4):
        fr, box = synth.npt_frame(system, f, strain_sigma=2e-3)
        cv, V, dV, F = run(ctx, fr, dev, box)
        ref = oracle.step_box(fr, oracle.make_params(box, n_cv=n_cv), c, w, sig, lattice=True)
        assert cv.shape == (n_cv + 3,)
        assert np.all(np.abs(cv - ref["s"]) <= TOL * np.abs(ref["s"]))
        assert np.array_equal(cv[n_cv:], box)  # the lattice CVs are the box, exactly
        assert abs(V - ref["V"]) <= TOL * max(abs(ref["V"]), 1.0)
        for d in range(n_cv + 3):
            assert abs(dV[d] - ref["dV"][d]) <= TOL * max(abs(ref["dV"][d]), 1.0 / sig[d])
        check_forces(F, ref["F"])
        check_box_grad(ctx.box_gradient(), ref["box_grad"], SIG_L[0])
        pairs = ctx.export_neighbors()
        assert np.array_equal(pairs, oracle.pairs_cells(fr, box, 3.5))
    ctx.close()


def test_virial_without_lattice_cvs(dev, system):
    c, w, sig = lattice_hills(system, 2, lattice=False)
    ctx = make_ctx(dev, system, 2, lattice=False, virial=True, hills=(c, w))
    fr = synth.perturbed_frame(system, 3)
    cv, V, dV, F = run(ctx, fr, dev)
    ref = oracle.step_box(fr, oracle.make_params(system.box, n_cv=2), c, w, sig, lattice=False)
    assert cv.shape == (2,)
    check_forces(F, ref["F"])
    check_box_grad(ctx.box_gradient(), ref["box_grad"], 0.02)
    # a scaled bias_forces scales the box gradient with it
    from paper_2510_06873_gb300 import metad
    Ft = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    metad.metad_bias_forces(ctx.ctx, Ft, False, -0.5)
    check_box_grad(ctx.box_gradient(), -0.5 * ref["box_grad"], 0.02)
    ctx.close()


def test_lattice_deposits(dev, system):
    c, w, sig = lattice_hills(system, 1, count=100)
    ctx = make_ctx(dev, system, 1, hills=(c, w))
    for f in range(5):
        fr, box = synth.npt_frame(system, 10 + f, strain_sigma=2e-3)
        run(ctx, fr, dev, box, deposit=True)
    cg, wg = ctx.get_hills()
    assert cg.shape == (105, 4)
    assert np.array_equal(cg[:100], c) and np.array_equal(wg[:100], w)
    # the oracle's own chain: each hill at the oracle's CVs of that frame
    live_c, live_w = c.copy(), w.copy()
    for f in range(5):
        fr, box = synth.npt_frame(system, 10 + f, strain_sigma=2e-3)
        s_ref = oracle.step_box(fr, oracle.make_params(box, n_cv=1), live_c, live_w, sig, lattice=True)["s"]
        h = oracle.deposit_sequence(np.vstack([live_c, s_ref[None, :]]), sig, 1.0, kbdt(), heights_prefix=live_w)[-1]
        live_c = np.vstack([live_c, s_ref[None, :]])
        live_w = np.append(live_w, h)
    assert np.all(np.abs(cg[100:] - live_c[100:]) <= TOL * np.abs(live_c[100:]))
    assert np.abs(wg - live_w).max() <= TOL
    ctx.close()


def test_cells_follow_the_box(dev, system):
    """Shrinking the box below a cell boundary lowers the cell count; growing
    it past the creation box keeps the allocated count (larger cells)."""
    ctx = make_ctx(dev, system, 1, hills=lattice_hills(system, 1, count=50)[:2])
    for scale in (0.9, 1.12, 1.0):
        box = system.box * scale
        fr = system.base.copy()
        fr[:, :3] = synth.wrap_to_box(system.base[:, :3].astype(np.float64) * scale, box)
        run(ctx, fr, dev, box)
        assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(fr, box, 3.5))
    ctx.close()


def test_rows_survive_small_box_changes(dev, system):
    """A slowly moving box keeps the Verlet rows (no rebuild) and the exact
    neighbour sets; a large jump rebuilds them."""
    ctx = make_ctx(dev, system, 1, hills=lattice_hills(system, 1, count=50)[:2])
    for f in range(6):
        fr, box = synth.npt_frame(system, f, strain_sigma=1e-3, period=400)
        run(ctx, fr, dev, box)
        assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(fr, box, 3.5))
    assert ctx.rebuild_count == 1  # the first step only
    box = system.box * 0.97
    fr = system.base.copy()
    fr[:, :3] = synth.wrap_to_box(system.base[:, :3].astype(np.float64) * 0.97, box)
    run(ctx, fr, dev, box)
    assert ctx.rebuild_count == 2
    assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(fr, box, 3.5))
    ctx.close()


def test_batched_lattice_systems_equal_single_steps(dev):
    from paper_2510_06873_gb300 import metad
    systems = [synth.wurtzite_system(n, cfg=8, sys=k) for k, n in enumerate((3000, 5000, 7000))]
    hills = [lattice_hills(s, 2, count=200) for s in systems]
    bat = [make_ctx(dev, s, 2, hills=h[:2]) for s, h in zip(systems, hills)]
    solo = [make_ctx(dev, s, 2, hills=h[:2]) for s, h in zip(systems, hills)]
    batch = metad.Batch(bat)
    for f in range(3):
        frames = [synth.npt_frame(s, f, strain_sigma=2e-3) for s in systems]
        pos = [torch.from_numpy(fr).to(dev) for fr, _ in frames]
        Fb = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
        Fs = [torch.zeros((s.n, 3), dtype=torch.float32, device=dev) for s in systems]
        for k in range(3):
            bat[k].set_box(frames[k][1])
            solo[k].set_box(frames[k][1])
        dep = np.array([f == 1, False, True], dtype=np.int32)
        batch.step(pos, Fb, deposit=dep)
        for k in range(3):
            solo[k].step(pos[k], Fs[k], deposit=bool(dep[k]))
            a, b = bat[k].read_results(), solo[k].read_results()
            assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
            assert torch.equal(Fb[k], Fs[k])
            assert np.array_equal(bat[k].box_gradient(), solo[k].box_gradient())
    batch.close()
    for c in bat + solo:
        c.close()


def test_lattice_errors(dev, system):
    from paper_2510_06873_gb300 import metad
    ctx = make_ctx(dev, system, 1)
    with pytest.raises(metad.MetadError) as e:
        ctx.box_gradient()
    assert e.value.status == metad.METAD_ERR_STATE
    with pytest.raises(metad.MetadError) as e:
        ctx.set_box([6.9, 40.0, 40.0])
    assert e.value.status == metad.METAD_ERR_INVALID
    ctx.close()
    plain = make_ctx(dev, system, 1, lattice=False)
    run(plain, system.base, dev)
    with pytest.raises(metad.MetadError) as e:
        plain.box_gradient()
    assert e.value.status == metad.METAD_ERR_INVALID
    plain.close()
    with pytest.raises(metad.MetadError):
        metad.Batch([make_ctx(dev, system, 1), make_ctx(dev, system, 1, lattice=False)])

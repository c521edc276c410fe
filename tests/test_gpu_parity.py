"""CUDA path against the FP64 oracle, through the C ABI (libmetad.so).

Neighbour sets must match bit for bit (as sorted pair lists); CVs, bias,
bias gradient and forces within the tolerances of parity_util.  Sizes span
several thread blocks with ragged tails; the 1M-atom case runs the launch
configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import TOL, check_bias, check_cv, check_forces, force_errors, kbdt, setup_hills

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RC = 3.5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06873_gb300 import build
    build.build()
    d = torch.device("cuda:0")
    # a non-default stream shared by torch's copies and the library's kernels
    torch.cuda.set_stream(torch.cuda.Stream(d))
    return d


def _metad():
    from paper_2510_06873_gb300 import metad
    return metad


def make_ctx(dev, system, mp, fp64=False, grid=None, hill_capacity=65536, max_nb=64, cn_unlike=True,
             sw=(6, 12), skin=1.0):
    metad = _metad()
    params = metad.params_for(system.n if hasattr(system, "n") else system[0], system.box, n_cv=mp.n_cv,
                              sigma=mp.sigma, fp64=fp64, grid=grid, hill_capacity=hill_capacity,
                              max_neighbors=max_nb, cn_unlike=cn_unlike, sw_n=sw[0], sw_m=sw[1],
                              stream=torch.cuda.current_stream(dev).cuda_stream, skin=skin)
    return metad.Metad(params)


def gpu_step(ctx, dev, frame, per_atom=False):
    pos = torch.from_numpy(np.ascontiguousarray(frame)).to(dev)
    F = torch.zeros((frame.shape[0], 3), dtype=torch.float32, device=dev)
    ctx.build_neighbors(pos)
    pa = torch.zeros((2, frame.shape[0]), dtype=torch.float64, device=dev) if per_atom else None
    s = ctx.cv_forward(per_atom=pa)
    V, dV = ctx.bias_eval()
    ctx.bias_forces(F)
    ctx.sync()
    out = {"s": s, "V": V, "dV": dV, "F": F.cpu().numpy().astype(np.float64)}
    if per_atom:
        out["per_atom"] = pa.cpu().numpy()
    return out


class _Sys:
    def __init__(self, pos, box):
        self.base = pos
        self.box = np.asarray(box, dtype=np.float64)
        self.n = pos.shape[0]
        self.sys = 0


# ------------------------------------------------------------------ neighbours
@pytest.mark.parametrize("lfac", [2.0, 2.2, 2.5, 3.0, 3.2, 4.0, 6.1])
def test_neighbours_bit_exact_small_boxes(dev, lfac):
    g = np.random.default_rng(int(lfac * 100))
    box = np.array([lfac * RC, (lfac + 0.37) * RC, (lfac + 0.71) * RC])
    n = 200 + int(lfac * 37)
    xyz = g.uniform(0.0, 1.0, (n, 3)) * box
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = synth.wrap_to_box(xyz, box)
    pos[:, 3] = (np.arange(n) % 2).astype(np.float32)
    s = _Sys(pos, box)
    mp = synth.MethodParams(n_cv=1, sigma=(0.05,))
    ctx = make_ctx(dev, s, mp, max_nb=128)
    ctx.build_neighbors(torch.from_numpy(pos).to(dev))
    got = ctx.export_neighbors()
    ref = oracle.pairs_brute(pos, box, RC)
    assert np.array_equal(got, ref)


def test_neighbours_guard_band_exact(dev):
    """Pairs placed within a few ulps of rc: the float32 estimate alone
    would misclassify some; the FP64 decision must match the definition."""
    g = np.random.default_rng(7)
    box = np.array([30.0, 30.0, 30.0])
    n = 400
    a = g.uniform(1.0, 28.0, (n // 2, 3))
    u = g.normal(size=(n // 2, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    b = a + u * RC * (1.0 + g.uniform(-3e-7, 3e-7, (n // 2, 1)))
    xyz = np.concatenate([a, b])
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = synth.wrap_to_box(xyz, box)
    s = _Sys(pos, box)
    ctx = make_ctx(dev, s, synth.MethodParams(n_cv=1, sigma=(0.05,)), max_nb=128)
    ctx.build_neighbors(torch.from_numpy(pos).to(dev))
    ref = oracle.pairs_brute(pos, box, RC)
    assert np.array_equal(ctx.export_neighbors(), ref)


@pytest.mark.parametrize("which", ["cfg1", "cfg2"])
def test_neighbours_bit_exact_configs(dev, which):
    system = synth.config1_system() if which == "cfg1" else synth.config2_system()
    frame = synth.perturbed_frame(system, 3)
    ctx = make_ctx(dev, system, synth.MethodParams(n_cv=1, sigma=(0.05,)))
    ctx.build_neighbors(torch.from_numpy(frame).to(dev))
    assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(frame, system.box, RC))


@pytest.mark.parametrize("skin", [0.0, 1.0])
def test_verlet_reuse_and_rebuild_stay_exact(dev, skin):
    """Frames within skin/2 of the last rebuild reuse the cell order and the
    Verlet rows; a larger move forces a rebuild; every exact row set equals
    the definition's."""
    system = synth.wurtzite_system(20000, cfg=95)
    ctx = make_ctx(dev, system, synth.MethodParams(n_cv=1, sigma=(0.05,)), skin=skin)
    frames = [synth.perturbed_frame(system, f) for f in range(3)]
    moved = frames[2].copy()
    moved[123, 0] = np.float32((float(moved[123, 0]) + 0.8) % system.box[0])  # > skin/2 from frame 0
    far = synth.perturbed_frame(system, 7, sigma=0.4)
    expect_rebuilds = [1, 1, 1, 2, 3] if skin > 0 else [1, 2, 3, 4, 5]
    for k, fr in enumerate(frames + [moved, far]):
        ctx.build_neighbors(torch.from_numpy(fr).to(dev))
        assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(fr, system.box, RC)), k
        assert ctx.rebuild_count == expect_rebuilds[k], (k, ctx.rebuild_count)


def test_drifting_trajectory_rebuilds_and_stays_exact(dev):
    """Whole steps along a drifting trajectory (random walk of 0.05 A per
    coordinate and frame on the thermal noise): the rows are rebuilt inside
    the run, and at sampled frames, rebuild or reuse, the neighbour set is
    the definition's bit for bit and the CVs, bias and forces match the
    oracle's."""
    system = synth.wurtzite_system(20000, cfg=95)
    mp = synth.MethodParams(n_cv=2, sigma=(0.05, 0.02))
    c, _ = setup_hills(system, mp, 300, cfg=95)
    ctx = make_ctx(dev, system, mp)
    ctx.deposit_hills(c)
    w = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    p = oracle.params_from(mp, system.box)
    F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    checked = []
    for f, frame in enumerate(synth.drift_trajectory(system, 36, step_sigma=0.05)):
        ctx.step(torch.from_numpy(frame).to(dev), F)
        if f % 7 == 6:
            assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(frame, system.box, RC)), f
            s, V, dV = ctx.read_results()
            ref = oracle.step(frame, p, c, w, mp.sigma)
            check_cv(s, ref["s"])
            check_bias(V, dV, ref["V"], ref["dV"], mp)
            check_forces(F.cpu().numpy().astype(np.float64), ref["F"])
            checked.append(ctx.rebuild_count)
    # the largest displacement since the last rebuild passes skin/2 = 0.5 A
    # every few frames at this step: several rebuilds, rows reused between
    assert 3 <= ctx.rebuild_count < 36, ctx.rebuild_count
    assert len(set(checked)) > 1


# ------------------------------------------------------------------ config 1 (FP64)
def test_config1_fp64_frames(dev):
    system = synth.config1_system()
    mp = synth.method_params(1)
    c, s_ref = setup_hills(system, mp, 200, cfg=1)
    ctx = make_ctx(dev, system, mp, fp64=True)
    w_gpu = ctx.deposit_hills(c)
    w_ref = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    assert np.allclose(w_gpu, w_ref, rtol=1e-13, atol=0)
    p = oracle.params_from(mp, system.box)
    for f in (0, 1, 57, 99):
        frame = synth.perturbed_frame(system, f)
        got = gpu_step(ctx, dev, frame, per_atom=True)
        ref = oracle.step(frame, p, c, w_ref, mp.sigma)
        check_cv(got["s"], ref["s"], tol=1e-12)
        check_bias(got["V"], got["dV"], ref["V"], ref["dV"], mp, tol=1e-12)
        # FP64 pairs, float32 force output: float32 rounding only
        check_forces(got["F"], ref["F"], tol=2e-7)
        _, cn, _ = oracle.cv(frame, p)
        assert np.allclose(got["per_atom"][0], cn, rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ config 2 (FP32 pairs)
def test_config2_frames(dev):
    system = synth.config2_system()
    mp = synth.method_params(2)
    c, s_ref = setup_hills(system, mp, 5000, cfg=2)
    ctx = make_ctx(dev, system, mp)
    w_gpu = ctx.deposit_hills(c)
    w_ref = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    assert np.allclose(w_gpu, w_ref, rtol=1e-12, atol=0)
    p = oracle.params_from(mp, system.box)
    for f in (0, 41, 99):
        frame = synth.perturbed_frame(system, f)
        got = gpu_step(ctx, dev, frame, per_atom=True)
        ref = oracle.step(frame, p, c, w_ref, mp.sigma)
        check_cv(got["s"], ref["s"])
        check_bias(got["V"], got["dV"], ref["V"], ref["dV"], mp)
        check_forces(got["F"], ref["F"])
        _, cn, q6 = oracle.cv(frame, p)
        assert np.max(np.abs(got["per_atom"][0] - cn)) <= 1e-5 * np.max(cn)
        assert np.max(np.abs(got["per_atom"][1] - q6)) <= 1e-5 * np.max(q6)


# ------------------------------------------------------------------ config 3 (1M, grid)
@pytest.mark.slow
def test_config3_neighbours_bit_exact(dev):
    """The 1M-atom neighbour set, as the benchmark's step uses it, against the
    oracle's cell search: the first frame (a rebuild), then a frame that
    reuses the rows (within skin/2), bit for bit as sorted pair lists."""
    system = synth.config3_system()
    mp = synth.method_params(3)
    ctx = make_ctx(dev, system, mp)
    F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    for f in (0, 499):
        frame = synth.perturbed_frame(system, f)
        ctx.step(torch.from_numpy(frame).to(dev), F)
        got = ctx.export_neighbors()
        ref = oracle.pairs_cells(frame, system.box, RC)
        print(f"frame {f}: {ref.shape[0]} pairs")
        assert np.array_equal(got, ref), f
    assert ctx.rebuild_count == 1
    ctx.close()


@pytest.mark.slow
def test_config3_grid_deposit_and_frames(dev):
    system = synth.config3_system()
    mp = synth.method_params(3)
    cfgp = synth.CONFIG_PARAMS[3]
    K1, K2 = cfgp["hills_folded"], cfgp["hills"]
    cen, s_ref = setup_hills(system, mp, K1 + K2, cfg=3)
    sig = np.asarray(mp.sigma)
    lo, hi = s_ref - 16 * sig, s_ref + 16 * sig
    # oracle: deposit, fold, deposit again
    w1 = oracle.deposit_sequence(cen[:K1], mp.sigma, mp.w0, kbdt(mp))
    G = oracle.HillGrid(cfgp["grid_n"], lo, hi)
    G.fold(cen[:K1], w1, mp.sigma)
    w2 = oracle.deposit_sequence(cen[K1:], mp.sigma, mp.w0, kbdt(mp), grid=G)
    # GPU
    ctx = make_ctx(dev, system, mp, grid=(cfgp["grid_n"], lo, hi))
    g1 = ctx.deposit_hills(cen[:K1])
    assert np.allclose(g1, w1, rtol=1e-12, atol=0)
    ctx.fold_hills()
    grid = ctx.get_grid()
    assert np.allclose(grid, G.data, rtol=1e-11, atol=1e-12 * np.max(np.abs(G.data)))
    g2 = ctx.deposit_hills(cen[K1:])
    assert np.allclose(g2, w2, rtol=1e-11, atol=0)
    p = oracle.params_from(mp, system.box)
    live_c, live_w = cen[K1:].copy(), w2.copy()
    for f in (0, 499):
        frame = synth.perturbed_frame(system, f)
        got = gpu_step(ctx, dev, frame)
        ref = oracle.step(frame, p, live_c, live_w, mp.sigma, grid=G)
        print(f"frame {f}: ds/s {(got['s'] - ref['s']) / ref['s']}, V {got['V']} vs {ref['V']}, "
              f"dV {got['dV']} vs {ref['dV']}, F err {force_errors(got['F'], ref['F'])}")
        check_cv(got["s"], ref["s"])
        check_bias(got["V"], got["dV"], ref["V"], ref["dV"], mp)
        check_forces(got["F"], ref["F"])
        if (f + 1) % cfgp["deposit_every"] == 0:
            # each side deposits at its own CVs; the heights differ through
            # the centres' CV difference only (well inside 1e-5)
            h = ctx.deposit_hill()
            href = oracle.deposit_sequence(np.vstack([live_c, ref["s"][None, :]]), mp.sigma, mp.w0, kbdt(mp),
                                           grid=G, heights_prefix=live_w)[-1]
            assert h == pytest.approx(href, rel=1e-5)
            live_c = np.vstack([live_c, ref["s"][None, :]])
            live_w = np.append(live_w, href)
    assert ctx.hill_count == K2 + 1


# ------------------------------------------------------------------ variants and edges
@pytest.mark.parametrize("n,fp64", [(1, False), (1, True), (2, False), (2, True), (129, False), (129, True),
                                    (1023, False), (1023, True), (4097, False), (4097, True)])
def test_ragged_and_tiny_systems(dev, n, fp64):
    """Ragged sizes around the block shape.

    Two atoms in FP32: the CVs are single rounded terms (one switch value,
    one averaged Q6 of a lone bond, exactly 1 in exact arithmetic), so their
    relative error is a few float32 roundings, ~1e-7, with nothing to average
    it out.  The CVs meet 1e-5; dV/ds need not: it moves by (d2V/ds2) ds,
    and 200 hills of width 0.02 within a few sigma give d2V/ds2 ~ V /
    sigma^2 ~ 1e4-1e5, so ds ~ 1e-7 shifts dV/ds by up to ~1e-3 against the
    floor 1e-5 w0 / sigma = 5e-4.  That is the CV's own float32 rounding
    amplified by the bias curvature, not an error of the bias or force
    arithmetic.  The test bounds it from the oracle alone: the CVs' rounding
    is at most 8 float32 ulps, the oracle's bias gradient and curvature
    (central differences of its bias at its own CVs) carry that to V and
    dV/ds, and the oracle's CV gradients (its forces for unit dV/ds) carry
    the dV/ds bound to the forces, each on top of the 1e-5 tolerance."""
    box = np.array([9.0, 9.5, 10.0]) * max(1.0, (n / 60.0) ** (1 / 3))
    if n <= 2:
        box = np.array([12.0, 12.0, 12.0])
        xyz = np.array([[1.0, 2.0, 3.0], [3.25, 2.5, 3.75]])[:n]
    else:
        g = np.random.default_rng(n)
        xyz = synth.rsa_fill(np.zeros((0, 3), np.float32), n, box, 0.0, box[0], 1.7, int(g.integers(1 << 62)))
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = xyz
    pos[:, 3] = (np.arange(n) % 2).astype(np.float32)
    s = _Sys(pos, box)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, box)
    s0, _, _ = oracle.cv(pos, p)
    c = synth.hill_centres(96, n, s0, mp.sigma, 200)
    ctx = make_ctx(dev, s, mp, fp64=fp64)
    ctx.deposit_hills(c)
    w = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    ref = oracle.step(pos, p, c, w, mp.sigma)
    got = gpu_step(ctx, dev, pos)
    if n == 1:
        assert np.all(got["s"] == 0.0) and np.all(got["F"] == 0.0)
        return
    if n == 2 and not fp64:
        check_cv(got["s"], ref["s"])
        sig = np.asarray(mp.sigma)
        ds = 8.0 * np.finfo(np.float32).eps * np.abs(ref["s"])  # the CVs' float32 rounding bound
        # the oracle's bias curvature by central differences at its own CVs
        H = np.zeros((2, 2))
        for d in range(2):
            e = np.zeros(2)
            e[d] = 1e-4 * sig[d]
            H[:, d] = (oracle.bias(ref["s"] + e, c, w, mp.sigma)[1] - oracle.bias(ref["s"] - e, c, w, mp.sigma)[1]) / (2 * e[d])
        tol_V = TOL * max(abs(ref["V"]), mp.w0) + np.abs(ref["dV"]) @ ds
        tol_dV = TOL * np.maximum(np.abs(ref["dV"]), mp.w0 / sig) + np.abs(H) @ ds
        assert abs(got["V"] - ref["V"]) <= tol_V, (got["V"], ref["V"], tol_V)
        assert np.all(np.abs(got["dV"] - ref["dV"]) <= tol_dV), (got["dV"], ref["dV"], tol_dV)
        # forces: the oracle's CV gradients (its forces for unit dV/ds) carry the dV/ds bound
        J = [np.abs(oracle.forces(pos, p, np.eye(2)[d])[0]) for d in range(2)]
        tol_F = tol_dV[0] * J[0] + tol_dV[1] * J[1] + TOL * np.abs(ref["F"]).max()
        assert np.all(np.abs(got["F"] - ref["F"]) <= tol_F)
        rel = [abs(got["dV"][d] - ref["dV"][d]) / max(abs(ref["dV"][d]), mp.w0 / mp.sigma[d]) for d in range(2)]
        print(f"N=2 FP32: ds/s {(got['s'] - ref['s']) / ref['s']}, dV/ds error over the floor {rel}")
        return
    tol = 1e-10 if fp64 else 1e-5
    check_cv(got["s"], ref["s"], tol=tol)
    check_bias(got["V"], got["dV"], ref["V"], ref["dV"], mp, tol=tol)
    check_forces(got["F"], ref["F"], tol=2e-7 if fp64 else 1e-5)


def test_isolated_atoms_have_zero_cv_and_force(dev):
    box = np.array([40.0, 40.0, 40.0])
    xyz = np.array([[5, 5, 5], [20, 20, 20], [33, 5, 20], [34.0, 6.0, 21.0], [10, 30, 30]], np.float64)
    pos = np.zeros((5, 4), np.float32)
    pos[:, :3] = xyz
    pos[:, 3] = [0, 1, 0, 1, 1]
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, box)
    ctx = make_ctx(dev, _Sys(pos, box), mp)
    s0, _, _ = oracle.cv(pos, p)
    c = np.array([s0 + np.array([0.01, 0.01]), s0 - np.array([0.02, 0.005])])
    ctx.deposit_hills(c)
    w = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    got = gpu_step(ctx, dev, pos, per_atom=True)
    ref = oracle.step(pos, p, c, w, mp.sigma)
    check_cv(got["s"], ref["s"])
    check_forces(got["F"], ref["F"])
    for k in (0, 1, 4):
        assert got["per_atom"][0][k] == 0.0 and got["per_atom"][1][k] == 0.0
        assert np.all(got["F"][k] == 0.0)


@pytest.mark.parametrize("variant", ["all_pairs", "switch_6_10", "unstretched_n1"])
def test_switch_and_mask_variants(dev, variant):
    system = synth.wurtzite_system(6000, cfg=91)
    frame = synth.perturbed_frame(system, 0)
    unlike, sw, ncv = True, (6, 12), 2
    if variant == "all_pairs":
        unlike = False
    elif variant == "switch_6_10":
        sw = (6, 10)
    else:
        ncv = 1
    mp = synth.MethodParams(n_cv=ncv, sigma=(0.05, 0.02)[:ncv], cn_unlike_only=unlike, sw_n=sw[0], sw_m=sw[1])
    p = oracle.make_params(system.box, mp.rc, mp.r0, sw[0], sw[1], True, unlike, ncv)
    s0, _, _ = oracle.cv(system.base, p)
    c = synth.hill_centres(91, 0, s0, mp.sigma, 300)
    ctx = make_ctx(dev, system, mp, cn_unlike=unlike, sw=sw)
    ctx.deposit_hills(c)
    w = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    got = gpu_step(ctx, dev, frame)
    ref = oracle.step(frame, p, c, w, mp.sigma)
    check_cv(got["s"], ref["s"])
    check_bias(got["V"], got["dV"], ref["V"], ref["dV"], mp)
    check_forces(got["F"], ref["F"])


def test_accumulate_scale_and_determinism(dev):
    system = synth.wurtzite_system(5000, cfg=92)
    frame = synth.perturbed_frame(system, 2)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, system.box)
    s0, _, _ = oracle.cv(system.base, p)
    c = synth.hill_centres(92, 0, s0, mp.sigma, 200)
    ctx = make_ctx(dev, system, mp)
    ctx.deposit_hills(c)
    pos = torch.from_numpy(frame).to(dev)
    F1 = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    F2 = torch.zeros_like(F1)
    ctx.step(pos, F1)
    ctx.step(pos, F2)
    ctx.sync()
    assert torch.equal(F1, F2)
    # the separate calls (sequential) give the step's bits (its hill kernel
    # runs concurrently with the adjoint on a side stream)
    F3 = torch.zeros_like(F1)
    ctx.build_neighbors(pos)
    ctx.cv_forward(want_host=False)
    ctx.bias_eval(want_host=False)
    ctx.bias_forces(F3)
    ctx.sync()
    assert torch.equal(F3, F1)
    base = torch.full_like(F1, 0.25)
    ctx.build_neighbors(pos)
    ctx.cv_forward(want_host=False)
    ctx.bias_eval(want_host=False)
    ctx.bias_forces(base, accumulate=True, scale=-2.0)
    ctx.sync()
    assert torch.allclose(base, 0.25 - 2.0 * F1, rtol=1e-6, atol=1e-9)


def test_host_step_equals_the_device_step(dev):
    """metad_step_host with page-locked host buffers, pageable ones, and
    page-locked ones off a 16-byte boundary gives the device step's bits,
    with and without accumulation into the caller's forces."""
    system = synth.wurtzite_system(5000, cfg=97)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, system.box)
    s0, _, _ = oracle.cv(system.base, p)
    ctx = make_ctx(dev, system, mp)
    ctx.deposit_hills(synth.hill_centres(97, 0, s0, mp.sigma, 200))
    frame = synth.perturbed_frame(system, 1)
    F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    ctx.step(torch.from_numpy(frame).to(dev), F)
    ctx.sync()
    ref = F.cpu().numpy()
    cv_ref, V_ref, _ = ctx.read_results()
    n = system.n

    def pinned(cols, offset):
        t = torch.zeros(n * cols + offset, dtype=torch.float32).pin_memory()
        return t.numpy()[offset:].reshape(n, cols)

    cases = {"page-locked": (pinned(4, 0), pinned(3, 0)),
             "pageable": (np.zeros((n, 4), np.float32), np.zeros((n, 3), np.float32)),
             "page-locked, 4-byte offset": (pinned(4, 1), pinned(3, 1))}
    for name, (ph, fh) in cases.items():
        ph[...] = frame
        fh[...] = 7.0
        cv, V = ctx.step_host(ph, fh)
        assert np.array_equal(fh, ref), name
        assert V == V_ref and np.array_equal(cv, cv_ref), name
        fh[...] = 0.5
        ctx.step_host(ph, fh, accumulate=True)
        assert np.array_equal(fh, np.float32(0.5) + ref), name
    ctx.close()


@pytest.mark.parametrize("fp64,skin", [(False, 1.0), (True, 1.0), (False, 2.0), (False, 0.0)])
def test_mirror_slots_equal_the_row_search(dev, fp64, skin):
    """The force pass finds each pair's slot in the higher atom's exact row
    from the mirror positions found at a rebuild (Verlet rows of at most 256
    entries), or by searching that row (larger rows).  Both give the same
    slots, so the same bits: 64 neighbours per atom (rows of up to 136
    Verlet entries at skin 1: mirror slots) against 128 (up to 272: the
    search), over frames that reuse the rows, frames that rebuild them, and
    an export of the neighbour list between a rebuild and the CV pass.  Skin
    2 gives rows of up to 248 entries, more than 32 of them j > i (positions
    past the first preloaded sector); skin 0 rebuilds every step (rows of 64
    and 128 entries: both contexts use mirror slots, found anew each step)."""
    system = synth.wurtzite_system(6000, cfg=93)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, system.box)
    s0, _, _ = oracle.cv(system.base, p)
    c = synth.hill_centres(93, 0, s0, mp.sigma, 200)
    ctxs = [make_ctx(dev, system, mp, fp64=fp64, skin=skin),
            make_ctx(dev, system, mp, fp64=fp64, max_nb=128, skin=skin)]
    for ctx in ctxs:
        ctx.deposit_hills(c, want_heights=False)
    w = oracle.deposit_sequence(c, mp.sigma, mp.w0, kbdt(mp))
    # small moves reuse the rows; sigma 0.4 moves atoms past skin / 2
    for f, sig in enumerate((0.05, 0.05, 0.4, 0.05, 0.4, 0.4, 0.05)):
        frame = synth.perturbed_frame(system, f, sigma=sig)
        pos = torch.from_numpy(frame).to(dev)
        out = []
        for ctx in ctxs:
            F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
            if f == 4:  # the filter runs for the export, the CV pass reuses its rows
                ctx.build_neighbors(pos)
                pairs = ctx.export_neighbors()
                ctx.cv_forward(want_host=False)
                ctx.bias_eval(want_host=False)
                ctx.bias_forces(F)
                assert np.array_equal(pairs, oracle.pairs_cells(frame, system.box, RC))
            else:
                ctx.step(pos, F)
            ctx.sync()
            out.append((F, ctx.read_results()))
        (Fa, ra), (Fb, rb) = out
        assert torch.equal(Fa, Fb), f
        assert np.array_equal(ra[0], rb[0]) and ra[1] == rb[1], f
    assert ctxs[0].rebuild_count == ctxs[1].rebuild_count >= (7 if skin == 0.0 else 4)
    ref = oracle.step(frame, p, c, w, mp.sigma)
    check_forces(Fa.cpu().numpy().astype(np.float64), ref["F"])
    for ctx in ctxs:
        ctx.close()


def test_graph_replay_matches_direct_steps(dev):
    """metad_step from a captured CUDA graph gives the direct launches' bits,
    through buffer changes (recapture), a deposit (the hill count changes)
    and an accumulate flag change."""
    system = synth.wurtzite_system(5000, cfg=94)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, system.box)
    s0, _, _ = oracle.cv(system.base, p)
    c = synth.hill_centres(94, 0, s0, mp.sigma, 300)
    direct = make_ctx(dev, system, mp)
    graph = make_ctx(dev, system, mp)
    graph.set_step_graph(True)
    direct.deposit_hills(c, want_heights=False)
    graph.deposit_hills(c, want_heights=False)
    frames = [torch.from_numpy(synth.perturbed_frame(system, f)).to(dev) for f in range(2)]
    FA = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    FB = torch.zeros_like(FA)
    launches0 = (direct.launch_count, graph.launch_count)
    for step in range(8):
        pos = frames[step % 2]
        dep = step == 3
        acc = step >= 6
        direct.step(pos, FA, accumulate=acc, deposit=dep)
        graph.step(pos, FB, accumulate=acc, deposit=dep)
        cvA, VA, _ = direct.read_results()
        cvB, VB, _ = graph.read_results()
        assert np.array_equal(cvA, cvB) and VA == VB, step
        assert torch.equal(FA, FB), step
    assert graph.hill_count == direct.hill_count == 301
    assert graph.launch_count - launches0[1] == direct.launch_count - launches0[0]


def test_graph_replay_with_new_buffers_every_step(dev):
    """A captured step serves new position and force buffers (patched into
    its nodes) with the direct launches' bits: a drifting trajectory, every
    frame in a buffer of its own, three force buffers in turn, a deposit
    and rebuilds on the way."""
    system = synth.wurtzite_system(5000, cfg=94)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, system.box)
    s0, _, _ = oracle.cv(system.base, p)
    c = synth.hill_centres(94, 0, s0, mp.sigma, 300)
    direct = make_ctx(dev, system, mp)
    graph = make_ctx(dev, system, mp)
    graph.set_step_graph(True)
    direct.deposit_hills(c, want_heights=False)
    graph.deposit_hills(c, want_heights=False)
    frames = [torch.from_numpy(f).to(dev) for f in synth.drift_trajectory(system, 14, step_sigma=0.1)]
    FA = [torch.zeros((system.n, 3), dtype=torch.float32, device=dev) for _ in range(3)]
    FB = [torch.zeros_like(FA[0]) for _ in range(3)]
    for step, pos in enumerate(frames):
        dep = step == 5
        direct.step(pos, FA[step % 3], deposit=dep)
        graph.step(pos, FB[step % 3], deposit=dep)
        cvA, VA, _ = direct.read_results()
        cvB, VB, _ = graph.read_results()
        assert np.array_equal(cvA, cvB) and VA == VB, step
        assert torch.equal(FA[step % 3], FB[step % 3]), step
    assert graph.rebuild_count == direct.rebuild_count > 2
    assert graph.hill_count == direct.hill_count == 301


def test_call_order_and_capacity_errors(dev):
    metad = _metad()
    system = synth.wurtzite_system(3000, cfg=93)
    frame = synth.perturbed_frame(system, 0)
    mp = synth.MethodParams(n_cv=2)
    ctx = make_ctx(dev, system, mp)
    F = torch.zeros((system.n, 3), dtype=torch.float32, device=dev)
    with pytest.raises(metad.MetadError) as e:
        ctx.cv_forward()
    assert e.value.status == metad.METAD_ERR_STATE
    with pytest.raises(metad.MetadError) as e:
        ctx.bias_forces(F)
    assert e.value.status == metad.METAD_ERR_STATE
    small = make_ctx(dev, system, mp, max_nb=4)
    small.build_neighbors(torch.from_numpy(frame).to(dev))
    with pytest.raises(metad.MetadError) as e:
        small.sync()
    assert e.value.status == metad.METAD_ERR_CAPACITY
    with pytest.raises(metad.MetadError) as e:
        small.build_neighbors(torch.from_numpy(frame).to(dev))
    assert e.value.status == metad.METAD_ERR_STATE
    full = make_ctx(dev, system, mp, hill_capacity=3)
    full.deposit_hills(np.zeros((3, 2)))
    with pytest.raises(metad.MetadError) as e:
        full.deposit_hill(np.zeros(2))
    assert e.value.status == metad.METAD_ERR_CAPACITY


def test_non_finite_position_reported(dev):
    metad = _metad()
    system = synth.wurtzite_system(3000, cfg=93)
    frame = synth.perturbed_frame(system, 0)
    frame[17, 1] = np.nan
    ctx = make_ctx(dev, system, synth.MethodParams(n_cv=2))
    ctx.build_neighbors(torch.from_numpy(frame).to(dev))
    with pytest.raises(metad.MetadError) as e:
        ctx.sync()
    assert e.value.status == metad.METAD_ERR_INVALID


def test_unwrapped_positions_are_wrapped(dev):
    system = synth.wurtzite_system(4000, cfg=94)
    frame = synth.perturbed_frame(system, 0)
    shifted = frame.copy()
    k = np.arange(system.n) % 3 == 0
    # whole-box shifts are exact in float32 for these magnitudes only when the
    # FP64 wrap reproduces the original coordinate; compare neighbour sets
    shifted[k, 0] = (frame[k, 0].astype(np.float64) + system.box[0]).astype(np.float32)
    wrapped = frame.copy()
    wrapped[:, :3] = synth.wrap_to_box(shifted[:, :3].astype(np.float64), system.box)
    ctx = make_ctx(dev, system, synth.MethodParams(n_cv=1, sigma=(0.05,)))
    ctx.build_neighbors(torch.from_numpy(shifted).to(dev))
    assert np.array_equal(ctx.export_neighbors(), oracle.pairs_cells(wrapped, system.box, RC))


def test_cv_trajectory_matches_oracle_and_single_frames(dev):
    """Offline CVs of a stored trajectory: each frame against the oracle, and
    bit for bit against stepping the frames one by one."""
    system = synth.wurtzite_system(20000, cfg=95)
    mp = synth.MethodParams(n_cv=2)
    p = oracle.params_from(mp, system.box)
    T = 6
    frames_h = np.stack([synth.perturbed_frame(system, f) for f in range(T)])
    frames = torch.from_numpy(frames_h).to(dev)
    ctx = make_ctx(dev, system, mp)
    cvs = ctx.cv_trajectory(frames)
    one = make_ctx(dev, system, mp)
    for t in range(T):
        ref, _, _ = oracle.cv(frames_h[t], p)
        check_cv(cvs[t], ref)
        one.build_neighbors(frames[t])
        assert np.array_equal(one.cv_forward(), cvs[t])


def test_fp32_reciprocals_against_correctly_rounded(dev):
    """The kernels' FP32 1/sqrt and 1/v (SFU estimate, one Newton-Raphson
    step with an exactly formed residual) against CUDA's correctly rounded
    intrinsics over the arguments the kernels see (squared pair distances,
    switch denominators): at most one ulp apart, almost always equal, and no
    rounding bias (the signed mean difference far below an ulp)."""
    metad = _metad()
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    for which, lo, hi in ((0, 0.25, 20.25), (2, 1.0, 12.0)):
        v = lo + (hi - lo) * torch.rand(4_000_000, generator=g, device=dev, dtype=torch.float32)
        mine, ref = torch.empty_like(v), torch.empty_like(v)
        metad.metad_probe_recip(v, mine, which, torch.cuda.current_stream(dev).cuda_stream)
        metad.metad_probe_recip(v, ref, which + 1, torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize(dev)
        ulps = (mine.view(torch.int32).long() - ref.view(torch.int32).long()).cpu().numpy()
        assert np.abs(ulps).max() <= 1, which
        assert np.mean(ulps != 0) < 1e-3, (which, np.mean(ulps != 0))
        assert abs(np.mean(ulps)) < 1e-4, (which, np.mean(ulps))
    # and the absolute error of the refined 1/sqrt against FP64
    v = 0.25 + 20.0 * torch.rand(1_000_000, generator=g, device=dev, dtype=torch.float32)
    mine = torch.empty_like(v)
    metad.metad_probe_recip(v, mine, 0, torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize(dev)
    exact = 1.0 / np.sqrt(v.double().cpu().numpy())
    rel = (mine.double().cpu().numpy() - exact) / exact
    assert np.abs(rel).max() <= 2.0 ** -23 and abs(rel.mean()) < 1e-9

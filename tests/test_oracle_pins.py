"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand, a wrong normalisation) fails at
least one of them:
  * neighbour sets: O(N^2) brute force by the definition, r == rc excluded;
  * switch: s(0) = 1, s(rc) = 0, s_raw(r0) = 1/2, the closed form 1/(1+x^6)
    and its derivative;
  * Y_6^m: scipy's independent spherical harmonics and finite differences;
  * CN: closed forms on perfect lattices and a two-atom system;
  * Q6: Steinhardt textbook values and the addition theorem (no Y_lm used);
  * bias (Eqs. 2-3): single-hill values and separability;
  * well-tempered heights: closed form for two hills at one centre;
  * grid: node reproduction and measured interpolation error;
  * forces: sum F = 0, zero torque on an isolated cluster, cubic point-group
    covariance, central finite differences of the full step.
"""
import math

import numpy as np
import pytest

import synth

RC = 3.5
KBDT = 0.0083144626 * 300.0 * (10.0 - 1.0)


def _pos4(xyz, species=None):
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    out = np.zeros((n, 4), dtype=np.float32)
    out[:, :3] = xyz
    out[:, 3] = 0.0 if species is None else species
    return out


def _lattice(basis, cell, reps, offset=(0.1, 0.2, 0.3), species=None):
    basis = np.asarray(basis, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    idx = np.stack(np.meshgrid(*[np.arange(r) for r in reps], indexing="ij"), -1).reshape(-1, 3)
    frac = (idx[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    box = cell * np.asarray(reps)
    xyz = (frac * cell + np.asarray(offset) * cell) % box
    sp = None
    if species is not None:
        sp = np.tile(np.asarray(species, dtype=np.float32), idx.shape[0])
    return _pos4(synth.wrap_to_box(xyz, box), sp), box


def _min_image(d, box):
    return d - box * np.round(d / box)


# ------------------------------------------------------------------ neighbours
@pytest.mark.parametrize("lfac", [2.0, 2.2, 2.5, 3.0, 3.2, 4.0])
def test_neighbour_cells_equal_bruteforce(oracle_mod, lfac):
    g = np.random.default_rng(int(lfac * 10))
    box = np.array([lfac * RC, (lfac + 0.37) * RC, (lfac + 0.71) * RC])
    n = 180
    xyz = g.uniform(0.0, 1.0, (n, 3)) * box
    pos = _pos4(synth.wrap_to_box(xyz, box))
    pb = oracle_mod.pairs_brute(pos, box, RC)
    pc = oracle_mod.pairs_cells(pos, box, RC)
    assert pb.shape[0] > 0
    assert np.array_equal(pb, pc)
    # sanity: pair count near N/2 * rho * 4/3 pi rc^3 for uniform points
    expect = 0.5 * n * (n / np.prod(box)) * 4.0 / 3.0 * math.pi * RC ** 3
    assert abs(pb.shape[0] - expect) < 0.2 * expect


def test_neighbour_predicate_strict_at_rc(oracle_mod):
    box = np.array([12.0, 12.0, 12.0])
    below = np.nextafter(np.float32(4.5), np.float32(0.0))
    pos = _pos4([[1.0, 1.0, 1.0], [4.5, 1.0, 1.0], [6.0, 6.0, 6.0], [6.0, 6.0, float(6.0 + 3.5)],
                 [9.0, 9.0, 1.0], [9.0, 9.0, float(below)]])
    pb = oracle_mod.pairs_brute(pos, box, RC)
    # 0-1 and 2-3 sit at exactly rc (excluded); 4-5 is just inside
    assert pb.tolist() == [[4, 5]]
    assert np.array_equal(pb, oracle_mod.pairs_cells(pos, box, RC))


def test_neighbour_minimum_image_across_boundary(oracle_mod):
    box = np.array([10.0, 10.0, 10.0])
    pos = _pos4([[0.2, 5.0, 5.0], [9.0, 5.0, 5.0], [5.0, 0.1, 9.9]])
    pb = oracle_mod.pairs_brute(pos, box, RC)
    assert pb.tolist() == [[0, 1]]


# ------------------------------------------------------------------ switch
def test_switch_closed_forms(oracle_mod):
    p = oracle_mod.make_params([10, 10, 10])
    pu = oracle_mod.make_params([10, 10, 10], stretch=False)
    r = np.array([0.0, 1.0, 2.0, 2.5, 3.0, 3.4999, 3.5, 4.0])
    s, ds = oracle_mod.switch(p, r)
    su, dsu = oracle_mod.switch(pu, r)
    x = r / 2.5
    # (1 - x^6) / (1 - x^12) = 1 / (1 + x^6)
    raw = 1.0 / (1.0 + x ** 6)
    src = 1.0 / (1.0 + 1.4 ** 6)
    assert src == pytest.approx(0.1172397, abs=1e-7)
    inside = r < RC
    assert np.allclose(su[inside], raw[inside], rtol=1e-13, atol=0)
    assert su[3] == pytest.approx(0.5, abs=1e-12)
    assert np.allclose(s[inside], (raw[inside] - src) / (1 - src), rtol=1e-12, atol=1e-15)
    assert s[0] == pytest.approx(1.0, abs=1e-15)
    assert s[6] == 0.0 and s[7] == 0.0 and ds[6] == 0.0
    assert abs(s[5]) < 1e-4
    dref = -6 * x ** 5 / (2.5 * (1 + x ** 6) ** 2) / (1 - src)
    assert np.allclose(ds[inside], dref[inside], rtol=1e-10, atol=1e-14)


def test_switch_derivative_fd_and_continuity(oracle_mod):
    p = oracle_mod.make_params([10, 10, 10], sw_n=6, sw_m=10)
    r = np.linspace(0.3, 3.4, 57)
    h = 1e-6
    sp, _ = oracle_mod.switch(p, r + h)
    sm, _ = oracle_mod.switch(p, r - h)
    _, ds = oracle_mod.switch(p, r)
    assert np.allclose((sp - sm) / (2 * h), ds, rtol=1e-6, atol=1e-9)
    # the x -> 1 branch joins the plain formula smoothly
    r1 = 2.5 * (1 + np.array([-2e-6, -0.9e-6, 0.0, 0.9e-6, 2e-6]))
    s1, d1 = oracle_mod.switch(p, r1)
    assert np.all(np.abs(np.diff(s1)) < 1e-5)
    assert np.allclose(d1, d1[2], rtol=1e-4)


# ------------------------------------------------------------------ Y_6^m
def test_ylm_matches_scipy_and_fd(oracle_mod):
    sp = pytest.importorskip("scipy.special")
    g = np.random.default_rng(3)
    d = g.normal(size=(40, 3)) * 2.0
    Y, G = oracle_mod.ylm6(d)
    r = np.linalg.norm(d, axis=1)
    theta = np.arccos(d[:, 2] / r)
    phi = np.arctan2(d[:, 1], d[:, 0])
    for mi, m in enumerate(range(-6, 7)):
        ref = sp.sph_harm_y(6, m, theta, phi)
        assert np.allclose(Y[:, mi], ref, rtol=0, atol=1e-12)
    # sum_m |Y|^2 = 13 / (4 pi)
    assert np.allclose(np.sum(np.abs(Y) ** 2, axis=1), 13 / (4 * math.pi), rtol=1e-13)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        Yp, _ = oracle_mod.ylm6(d + e)
        Ym, _ = oracle_mod.ylm6(d - e)
        assert np.allclose((Yp - Ym) / (2 * h), G[:, :, a], rtol=1e-6, atol=1e-8)


# ------------------------------------------------------------------ CN
def test_cn_rocksalt_simple_cubic(oracle_mod):
    a = 2.6  # first shell 2.6 < rc < second shell 3.677
    pos, box = _lattice([[0, 0, 0]], [a, a, a], (6, 6, 6))
    idx = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos[:, 3] = (idx.sum(1) % 2).astype(np.float32)
    for unlike in (True, False):
        p = oracle_mod.make_params(box, cn_unlike_only=unlike, n_cv=1)
        s, cn, _ = oracle_mod.cv(pos, p)
        sa, _ = oracle_mod.switch(p, [a])
        assert np.allclose(cn, 6 * sa[0], rtol=1e-6)
        assert s[0] == pytest.approx(6 * sa[0], rel=1e-6)


def test_cn_like_species_masked(oracle_mod):
    a = 2.6
    pos, box = _lattice([[0, 0, 0]], [a, a, a], (4, 4, 4))
    pos[:, 3] = 1.0  # all one species
    p = oracle_mod.make_params(box, cn_unlike_only=True, n_cv=1)
    s, cn, _ = oracle_mod.cv(pos, p)
    assert s[0] == 0.0 and np.all(cn == 0.0)


def test_two_atom_cn_and_force(oracle_mod):
    box = np.array([10.0, 10.0, 10.0])
    pos = _pos4([[2.0, 3.0, 4.0], [4.25, 3.5, 4.75]], [0.0, 1.0])
    p = oracle_mod.make_params(box, n_cv=1)
    d = pos[1, :3].astype(np.float64) - pos[0, :3].astype(np.float64)
    r = np.linalg.norm(d)
    sr, dsr = oracle_mod.switch(p, [r])
    s, _, _ = oracle_mod.cv(pos, p)
    assert s[0] == pytest.approx(sr[0], rel=1e-14)  # (1/N) * 2 * s(r) with N = 2
    V1 = 1.7
    F, _ = oracle_mod.forces(pos, p, [V1])
    # F_0 = -V1 ds1/dr_0 = V1 s'(r) d / r ; F_1 = -F_0
    assert np.allclose(F[0], V1 * dsr[0] * d / r, rtol=1e-12)
    assert np.allclose(F[1], -F[0], rtol=1e-14)


# ------------------------------------------------------------------ Q6
def _steinhardt_from_addition(vectors):
    u = vectors / np.linalg.norm(vectors, axis=1)[:, None]
    t = np.clip(u @ u.T, -1, 1)
    p6 = (231 * t ** 6 - 315 * t ** 4 + 105 * t ** 2 - 5) / 16
    n = u.shape[0]
    return math.sqrt(p6.sum() / n ** 2)


LATTICES = {
    # name: (basis, cell, reps, nearest-neighbour vectors, textbook Q6)
    "sc": ([[0, 0, 0]], [2.5, 2.5, 2.5], (5, 5, 5), None, math.sqrt(1 / 8)),
    "fcc": ([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], [2.5 * math.sqrt(2)] * 3, (4, 4, 4), None, 0.57452),
    "diamond": ([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5], [0.25, 0.25, 0.25], [0.75, 0.75, 0.25],
                 [0.75, 0.25, 0.75], [0.25, 0.75, 0.75]], [2.5 * 4 / math.sqrt(3)] * 3, (3, 3, 3), None, 0.62854),
    "hcp": ([[0, 0, 0], [0.5, 0.5, 0], [0.5, 1 / 6, 0.5], [0, 2 / 3, 0.5]],
            [2.5, 2.5 * math.sqrt(3), 2.5 * math.sqrt(8 / 3)], (5, 3, 3), None, 0.48476),
}


@pytest.mark.parametrize("name", sorted(LATTICES))
def test_q6_textbook_lattices(oracle_mod, name):
    basis, cell, reps, _, ref = LATTICES[name]
    pos, box = _lattice(basis, cell, reps)
    p = oracle_mod.make_params(box, n_cv=2)
    s, cn, q6 = oracle_mod.cv(pos, p)
    # nearest-neighbour shell straight from the geometry, Q6 by the addition theorem
    x = pos[:, :3].astype(np.float64)
    d = _min_image(x - x[0], box)
    r = np.linalg.norm(d, axis=1)
    shell = (r > 0.1) & (r < RC)
    q6_add = _steinhardt_from_addition(d[shell])
    assert q6_add == pytest.approx(ref, abs=6e-6)
    # equal weights within float32 rounding of the lattice sites
    assert np.allclose(q6, q6_add, rtol=2e-6)
    assert s[1] == pytest.approx(q6_add, rel=2e-6)


def test_q6_addition_theorem_every_atom(oracle_mod):
    """qbar6(i)^2 = sum_ab c_a c_b P6(u_a . u_b) over every direction entering
    qbar(i), with weights from the switch: independent of Y_lm entirely."""
    s = synth.rsa_liquid_system(150, 0.06, 1.7, cfg=90, sys=1)
    pos, box = s.base, s.box
    p = oracle_mod.make_params(box, n_cv=2)
    _, _, q6 = oracle_mod.cv(pos, p)
    pairs = oracle_mod.pairs_brute(pos, box, RC)
    n = pos.shape[0]
    x = pos[:, :3].astype(np.float64)
    nb = [[] for _ in range(n)]
    for i, j in pairs:
        d = _min_image(x[j] - x[i], box)
        w, _ = oracle_mod.switch(p, [np.linalg.norm(d)])
        nb[i].append((j, w[0], d))
        nb[j].append((i, w[0], -d))
    W = np.array([sum(e[1] for e in nb[i]) for i in range(n)])
    for i in range(n):
        coef, vecs = [], []
        for j, w, d in nb[i]:
            coef.append(w / (W[i] * (1 + W[i])))
            vecs.append(d)
            for k, w2, d2 in nb[j]:
                coef.append(w / (1 + W[i]) * w2 / W[j])
                vecs.append(d2)
        if not coef:
            assert q6[i] == 0.0
            continue
        c = np.array(coef)
        u = np.array(vecs)
        u = u / np.linalg.norm(u, axis=1)[:, None]
        t = np.clip(u @ u.T, -1, 1)
        p6 = (231 * t ** 6 - 315 * t ** 4 + 105 * t ** 2 - 5) / 16
        ref = math.sqrt(max(c @ p6 @ c, 0.0))
        assert q6[i] == pytest.approx(ref, rel=1e-11, abs=1e-14)


# ------------------------------------------------------------------ bias
def test_single_hill_values(oracle_mod):
    c = np.array([[0.3, 0.7]])
    w = np.array([1.3])
    sig = np.array([0.05, 0.02])
    V, dV = oracle_mod.bias(c[0], c, w, sig)
    assert V == pytest.approx(1.3, rel=1e-15) and np.all(dV == 0.0)
    for d in range(2):
        s = c[0].copy()
        s[d] += sig[d]
        V, dV = oracle_mod.bias(s, c, w, sig)
        assert V == pytest.approx(1.3 * math.exp(-0.5), rel=1e-14)
        assert dV[d] == pytest.approx(-1.3 * math.exp(-0.5) / sig[d], rel=1e-13)
    # 2-D hill = product of two 1-D hills
    g = np.random.default_rng(5)
    for _ in range(5):
        s = c[0] + g.normal(size=2) * sig
        V, _ = oracle_mod.bias(s, c, w, sig)
        V0, _ = oracle_mod.bias(s[:1], c[:, :1], np.ones(1), sig[:1])
        V1, _ = oracle_mod.bias(s[1:], c[:, 1:], np.ones(1), sig[1:])
        assert V == pytest.approx(1.3 * V0 * V1, rel=1e-13)


def test_bias_gradient_fd(oracle_mod):
    g = np.random.default_rng(6)
    sig = np.array([0.05, 0.02])
    c = g.normal(size=(50, 2)) * sig * 3 + np.array([2.0, 0.4])
    w = g.uniform(0.2, 1.0, 50)
    s = np.array([2.01, 0.405])
    _, dV = oracle_mod.bias(s, c, w, sig)
    for d in range(2):
        h = 1e-6 * sig[d]
        e = np.zeros(2)
        e[d] = h
        Vp, _ = oracle_mod.bias(s + e, c, w, sig)
        Vm, _ = oracle_mod.bias(s - e, c, w, sig)
        assert (Vp - Vm) / (2 * h) == pytest.approx(dV[d], rel=1e-7, abs=1e-9)


def test_well_tempered_heights(oracle_mod):
    sig = np.array([0.05])
    w = oracle_mod.deposit_sequence(np.array([[1.0], [1.0]]), sig, 1.0, KBDT)
    assert KBDT == pytest.approx(22.44905, abs=1e-5)
    assert w[0] == 1.0
    assert w[1] == pytest.approx(math.exp(-1.0 / KBDT), rel=1e-14)
    assert w[1] == pytest.approx(0.956433, abs=1e-6)
    far = oracle_mod.deposit_sequence(np.array([[1.0], [1.0], [3.0]]), sig, 1.0, KBDT)
    assert far[2] == pytest.approx(1.0, abs=1e-300)
    # three at one centre: w3 = exp(-(1 + w2)/kBdT)
    w3 = oracle_mod.deposit_sequence(np.array([[0.0, 0.0]] * 3), np.array([0.05, 0.02]), 1.0, KBDT)
    assert w3[2] == pytest.approx(math.exp(-(1.0 + w3[1]) / KBDT), rel=1e-14)


# ------------------------------------------------------------------ grid
def test_grid_reproduces_nodes_and_bounds_error(oracle_mod):
    sig = np.array([0.05, 0.02])
    g = np.random.default_rng(8)
    ctr = np.array([2.0, 0.4])
    K = 300
    c = ctr + (g.uniform(size=(K, 2)) * 2 - 1) * 10 * sig
    w = g.uniform(0.1, 1.0, K)
    lo, hi = ctr - 16 * sig, ctr + 16 * sig
    G = oracle_mod.HillGrid((200, 200), lo, hi)
    G.fold(c, w, sig)
    h = (hi - lo) / 199
    for a, b in [(0, 0), (17, 133), (100, 100), (199, 199), (198, 1)]:
        s = np.array([lo[0] + a * h[0], lo[1] + b * h[1]])
        V, dV = oracle_mod.bias(s, np.zeros((0, 2)), np.zeros(0), sig, grid=G)
        Ve, dVe = oracle_mod.bias(s, c, w, sig)
        assert V == pytest.approx(G.data[a, b, 0], rel=1e-12, abs=1e-14)
        assert np.allclose(dV, G.data[a, b, 1:3], rtol=1e-10, atol=1e-10)
        assert V == pytest.approx(Ve, rel=1e-12, abs=1e-14)
        assert np.allclose(dV, dVe, rtol=1e-10, atol=1e-9)
    probes = lo + g.uniform(size=(1000, 2)) * (hi - lo)
    errV, errG, Vmax = 0.0, 0.0, 0.0
    for s in probes:
        V, dV = oracle_mod.bias(s, np.zeros((0, 2)), np.zeros(0), sig, grid=G)
        Ve, dVe = oracle_mod.bias(s, c, w, sig)
        errV = max(errV, abs(V - Ve))
        errG = max(errG, np.max(np.abs((dV - dVe) * sig)))
        Vmax = max(Vmax, Ve)
    # bicubic Hermite at h = 0.16 sigma: measured ~1e-5 of the bias scale
    assert errV < 1e-4 * Vmax
    assert errG < 2e-3 * Vmax
    # outside the range the grid adds nothing
    V, dV = oracle_mod.bias(hi + sig, np.zeros((0, 2)), np.zeros(0), sig, grid=G)
    assert V == 0.0 and np.all(dV == 0.0)


# ------------------------------------------------------------------ forces
def _small_system(n=60, L=9.0, seed=11, dmin=1.6):
    box = np.array([L, L + 0.3, L + 0.6])
    g = np.random.default_rng(seed)
    xyz = synth.rsa_fill(np.zeros((0, 3), np.float32), n, box, 0.0, box[0], dmin, int(g.integers(1 << 62)))
    sp = np.zeros(n, dtype=np.float32)
    sp[n // 2:] = 1.0
    return _pos4(xyz, g.permutation(sp)), box


def _hills_near(s, sig, k, seed):
    g = np.random.default_rng(seed)
    c = np.asarray(s)[None, :] + g.normal(size=(k, len(s))) * np.asarray(sig)[None, :] * 1.5
    return c, g.uniform(0.5, 1.5, k)


@pytest.mark.parametrize("n_cv,unlike", [(1, True), (1, False), (2, True)])
def test_forces_central_differences(oracle_mod, n_cv, unlike):
    pos, box = _small_system()
    p = oracle_mod.make_params(box, n_cv=n_cv, cn_unlike_only=unlike)
    sig = np.array([0.05, 0.02])[:n_cv]
    s0, _, _ = oracle_mod.cv(pos, p)
    c, w = _hills_near(s0, sig, 12, 2)
    out = oracle_mod.step(pos, p, c, w, sig)
    F = out["F"]
    g = np.random.default_rng(4)
    worst = 0.0
    for i in g.choice(pos.shape[0], 12, replace=False):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] = np.float32(pos[i, a] + np.float32(1.0 / 16384))
            pm[i, a] = np.float32(pos[i, a] - np.float32(1.0 / 16384))
            h2 = float(pp[i, a]) - float(pm[i, a])
            Vp = oracle_mod.step(pp, p, c, w, sig)["V"]
            Vm = oracle_mod.step(pm, p, c, w, sig)["V"]
            fd = -(Vp - Vm) / h2
            worst = max(worst, abs(fd - F[i, a]))
    assert worst < 1e-6 * np.max(np.abs(F)) + 1e-12


def test_forces_sum_to_zero_and_torque_free(oracle_mod):
    pos, box = _small_system(n=90, L=10.0, seed=12)
    p = oracle_mod.make_params(box, n_cv=2)
    F, _ = oracle_mod.forces(pos, p, [0.7, -2.3])
    assert np.max(np.abs(F.sum(0))) < 1e-13 * np.max(np.abs(F)) * pos.shape[0]
    # isolated cluster in a large box: no periodic images, so sum r x F = 0
    g = np.random.default_rng(13)
    xyz = synth.rsa_fill(np.zeros((0, 3), np.float32), 40, np.array([9.0, 9.0, 9.0]), 0.0, 9.0, 1.6,
                         int(g.integers(1 << 62))).astype(np.float64) + 20.0
    cl = _pos4(xyz, (np.arange(40) % 2).astype(np.float32))
    bigbox = np.array([50.0, 50.0, 50.0])
    pc = oracle_mod.make_params(bigbox, n_cv=2)
    F, _ = oracle_mod.forces(cl, pc, [0.7, -2.3])
    x = cl[:, :3].astype(np.float64)
    torque = np.cross(x - x.mean(0), F).sum(0)
    assert np.max(np.abs(torque)) < 1e-12 * np.max(np.abs(F)) * 40 * 10


def test_cubic_point_group_covariance(oracle_mod):
    L = 10.0
    box = np.array([L, L, L])
    g = np.random.default_rng(21)
    xyz = synth.rsa_fill(np.zeros((0, 3), np.float32), 70, box, 0.0, L, 1.6, int(g.integers(1 << 62)))
    # coordinates on a 2^-10 grid inside (0, L): x -> L - x is then exact in float32
    xyz = np.clip(np.round(xyz.astype(np.float64) * 1024.0) / 1024.0, 1.0 / 1024, L - 1.0 / 1024).astype(np.float32)
    sp = (np.arange(70) % 2).astype(np.float32)
    pos = _pos4(xyz, sp)
    p = oracle_mod.make_params(box, n_cv=2)
    s0, cn0, q0 = oracle_mod.cv(pos, p)
    F0, _ = oracle_mod.forces(pos, p, [0.4, 1.1])
    import itertools
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product([1, -1], repeat=3):
            R = np.zeros((3, 3))
            for a in range(3):
                R[a, perm[a]] = flips[a]
            x = pos[:, :3].astype(np.float64) @ R.T
            x = np.where(x < 0, x + L, x)  # exact for float32 values in (0, L)
            q = _pos4(x.astype(np.float32), sp)
            assert np.array_equal(q[:, :3].astype(np.float64), x)
            s, cn, q6 = oracle_mod.cv(q, p)
            assert np.allclose(s, s0, rtol=1e-12)
            assert np.allclose(q6, q0, rtol=1e-11, atol=1e-14)
            F, _ = oracle_mod.forces(q, p, [0.4, 1.1])
            assert np.allclose(F, F0 @ R.T, rtol=1e-9, atol=1e-12 * np.max(np.abs(F0)))


# ------------------------------------------------------------------ generator
def test_generator_shapes_and_constraints():
    s = synth.config1_system()
    assert s.n == 1000 and s.box[0] == pytest.approx((1000 / 0.08) ** (1 / 3))
    assert np.all(s.base[:, :3] >= 0) and np.all(s.base[:, :3].astype(np.float64) < s.box)
    assert int(s.base[:, 3].sum()) == 500
    f0 = synth.perturbed_frame(s, 0)
    f0b = synth.perturbed_frame(s, 0)
    assert np.array_equal(f0, f0b)
    d = f0[:, :3].astype(np.float64) - s.base[:, :3]
    d = d - s.box * np.round(d / s.box)
    assert 0.04 < d.std() < 0.06


# ------------------------------------------------------------------ free energy
def test_fes_points_single_hill_closed_form(oracle_mod):
    """One hill: F(s) - F_min = gamma/(gamma-1) w (1 - exp(-(s-c)^2/2sigma^2)) over
    points that include the centre (where F is lowest)."""
    c = np.array([[1.0, 0.3]])
    w = np.array([2.5])
    sig = np.array([0.05, 0.02])
    gamma = 10.0
    pts = np.array([[1.0, 0.3], [1.05, 0.3], [1.0, 0.32], [1.1, 0.26]])
    F = oracle_mod.fes_points(pts, c, w, sig, gamma)
    e = np.exp(-((pts - c[0]) ** 2 / (2 * sig ** 2)).sum(axis=1))
    assert np.allclose(F, gamma / (gamma - 1) * w[0] * (1 - e), rtol=1e-13, atol=1e-14)


def test_fes_reweight_unbiased_is_log_histogram(oracle_mod):
    """With V = 0 the reweighted F is -(1/beta) log of the plain histogram
    fractions (numpy's histogram as the independent count)."""
    g = np.random.default_rng(11)
    S = np.column_stack([g.normal(1.0, 0.2, 4000), g.normal(0.3, 0.05, 4000)])
    lo, hi, n = (0.2, 0.1), (1.8, 0.5), (8, 5)
    beta = 1 / 2.494
    F = oracle_mod.fes_reweight(S, np.zeros(len(S)), beta, lo, hi, n)
    H, _, _ = np.histogram2d(S[:, 0], S[:, 1], bins=n, range=[(lo[0], hi[0]), (lo[1], hi[1])])
    P = H.ravel() / H.sum()
    ref = np.full(P.size, np.inf)
    ref[P > 0] = -np.log(P[P > 0]) / beta
    ref[P > 0] -= ref[P > 0].min()
    assert np.array_equal(np.isinf(F), np.isinf(ref))
    fin = ~np.isinf(F)
    assert np.allclose(F[fin], ref[fin], rtol=1e-12, atol=1e-12)


def test_fes_reweight_weights_and_shift_invariance(oracle_mod):
    """Two bins, samples with known biases: F difference is -(1/beta) log of
    the weight ratio; a constant added to every V changes nothing."""
    beta = 0.5
    S = np.array([[0.1], [0.1], [0.7]])
    V = np.array([0.0, 2.0, 1.0])
    F = oracle_mod.fes_reweight(S, V, beta, (0.0,), (1.0,), (2,))
    w0 = np.exp(beta * 0.0) + np.exp(beta * 2.0)
    w1 = np.exp(beta * 1.0)
    assert abs((F[1] - F[0]) - (-(1 / beta) * np.log(w1 / w0))) < 1e-13
    F2 = oracle_mod.fes_reweight(S, V + 7.5, beta, (0.0,), (1.0,), (2,))
    assert np.allclose(F, F2, rtol=0, atol=1e-13)

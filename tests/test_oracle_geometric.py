"""Pins for the oracle of the small-system CVs (torsions, nearest distance)
and the periodic hills, against facts fixed by geometry and mathematics:
  * torsion: a construction whose angle is known by design (any rotation,
    translation, bond lengths, across box faces), the IUPAC sign (mirror
    image flips it), cis 0 / trans pi, collinear atoms;
  * its gradient (Blondel-Karplus form): central differences, zero net force
    and torque;
  * nearest distance: hand-placed candidates (exact distances), the minimum
    image, ties, the soft minimum's closed forms and bounds, central
    differences;
  * periodic hills: a hill across the -pi/pi seam, heights deposited across
    it, and the full step's forces against differences of its energy.
"""
import math

import numpy as np
import pytest

import synth

oracle = pytest.importorskip("oracle")
from oracle import geometric as og  # noqa: E402


def _rot(g):
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def _quad_with_angle(theta, g):
    """Four points whose dihedral about the b -> c axis is theta by design:
    b at 0, c on +z, a in the xz half-plane x > 0, d at azimuth theta."""
    h = g.uniform(1.2, 1.8)
    ra, rd = g.uniform(0.8, 1.5, 2)
    a = np.array([ra, 0.0, g.uniform(-0.8, 0.8)])
    d = np.array([rd * math.cos(theta), rd * math.sin(theta), h + g.uniform(-0.8, 0.8)])
    return np.array([a, [0.0, 0.0, 0.0], [0.0, 0.0, h], d])


def _frame(xyz, box, dtype=np.float32):
    out = np.zeros((len(xyz), 4), dtype=dtype)
    out[:, :3] = np.mod(xyz, box) if dtype == np.float32 else xyz
    return out


def _ang_close(x, y, tol):
    return abs(math.remainder(x - y, 2 * math.pi)) <= tol


@pytest.mark.parametrize("theta", np.linspace(-math.pi + 0.05, math.pi - 0.05, 13))
def test_torsion_equals_constructed_angle(theta):
    g = np.random.default_rng(11)
    box = np.array([9.0, 10.0, 11.0])
    for _ in range(5):
        p = _quad_with_angle(theta, g) @ _rot(g).T + g.uniform(-20, 20, 3)  # crosses faces after wrapping
        f = _frame(p, box)
        assert _ang_close(og.torsion(f, box, (0, 1, 2, 3)), theta, 2e-5)
        # the mirror image has the opposite angle
        m = p.copy()
        m[:, 0] *= -1.0
        assert _ang_close(og.torsion(_frame(m, box), box, (0, 1, 2, 3)), -theta, 2e-5)
        # reversing the atom order keeps it
        assert _ang_close(og.torsion(f, box, (3, 2, 1, 0)), theta, 2e-5)


def test_torsion_cis_trans_and_collinear():
    box = np.array([20.0, 20.0, 20.0])
    cis = _frame(np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1.5], [1, 0, 1.5]]) + 5.0, box)
    trans = _frame(np.array([[1, 0, 0], [0, 0, 0], [0, 0, 1.5], [-1, 0, 1.5]]) + 5.0, box)
    assert og.torsion(cis, box, (0, 1, 2, 3)) == 0.0
    assert abs(abs(og.torsion(trans, box, (0, 1, 2, 3))) - math.pi) < 1e-12
    line = _frame(np.array([[0, 0, -1.0], [0, 0, 0], [0, 0, 1.5], [1, 0, 1.5]]) + 5.0, box)
    assert og.torsion(line, box, (0, 1, 2, 3)) == 0.0
    assert not np.any(og.torsion_grad(line, box, (0, 1, 2, 3)))


def test_torsion_gradient_fd_force_and_torque_free():
    g = np.random.default_rng(5)
    box = np.array([50.0, 50.0, 50.0])
    for _ in range(20):
        p = g.normal(0.0, 1.0, (4, 3)) + 25.0
        f = _frame(p, box, np.float64)
        gr = og.torsion_grad(f, box, (0, 1, 2, 3))
        h = 1e-6
        for i in range(4):
            for a in range(3):
                fp, fm = f.copy(), f.copy()
                fp[i, a] += h
                fm[i, a] -= h
                fd = math.remainder(og.torsion(fp, box, (0, 1, 2, 3)) - og.torsion(fm, box, (0, 1, 2, 3)),
                                    2 * math.pi) / (2 * h)
                assert abs(fd - gr[i, a]) <= 1e-6 * max(1.0, abs(gr[i, a]))
        assert np.abs(gr.sum(axis=0)).max() < 1e-12 * np.abs(gr).max() * 10
        torque = sum(np.cross(p[i] - 25.0, gr[i]) for i in range(4))
        assert np.abs(torque).max() < 1e-10 * np.abs(gr).max() * 10


def test_nearest_distance_hand_placed_and_minimum_image():
    box = np.array([12.0, 12.0, 12.0])
    xyz = np.array([[6, 6, 6], [8, 6, 6], [6, 7.5, 6], [6, 6, 9], [6, 6, 6 - 1.25]])
    f = _frame(xyz, box)
    s, gr = og.nearest_distance(f, box, 0, [1, 2, 3, 4])
    assert s == 1.0 + 0.25 and set(gr) == {0, 4}
    assert np.array_equal(gr[4], [0, 0, -1]) and np.array_equal(gr[0], [0, 0, 1])
    # a candidate across the face is nearer by the minimum image
    xyz2 = np.array([[0.5, 6, 6], [11.7, 6, 6], [3.0, 6, 6]])
    s2, gr2 = og.nearest_distance(_frame(xyz2, box), box, 0, [1, 2])
    assert abs(s2 - 0.8) < 1e-6 and set(gr2) == {0, 1}
    assert gr2[1][0] == -1.0  # the image lies at -x
    # a tie goes to the first candidate in list order
    xyz3 = np.array([[6, 6, 6], [7, 6, 6], [5, 6, 6]])
    _, gr3 = og.nearest_distance(_frame(xyz3, box), box, 0, [2, 1])
    assert set(gr3) == {0, 2}


def test_soft_minimum_closed_forms_and_bounds():
    box = np.array([20.0, 20.0, 20.0])
    one = _frame(np.array([[5, 5, 5], [7, 5, 5]]), box)
    assert og.nearest_distance(one, box, 0, [1], beta=7.0)[0] == 2.0
    # k candidates at one distance: s = r - log(k) / beta
    for k in (2, 3, 6):
        dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]])[:k]
        f = _frame(np.vstack([[10, 10, 10], 10 + 1.5 * dirs]), box)
        s, gr = og.nearest_distance(f, box, 0, list(range(1, k + 1)), beta=4.0)
        assert abs(s - (1.5 - math.log(k) / 4.0)) < 1e-14
        assert np.abs(gr[0]).max() < 1e-15 or k == 3  # symmetric sets pull the reference nowhere
    g = np.random.default_rng(3)
    f = _frame(g.uniform(0, 20, (40, 3)), box)
    exact = og.nearest_distance(f, box, 0, range(1, 40))[0]
    for beta in (1.0, 10.0, 100.0):
        s = og.nearest_distance(f, box, 0, range(1, 40), beta=beta)[0]
        assert exact - math.log(39) / beta - 1e-12 <= s <= exact + 1e-12
    assert abs(og.nearest_distance(f, box, 0, range(1, 40), beta=1e4)[0] - exact) < 1e-3


@pytest.mark.parametrize("beta", [0.0, 3.0])
def test_nearest_distance_gradient_fd(beta):
    g = np.random.default_rng(9)
    box = np.array([15.0, 15.0, 15.0])
    f = _frame(g.uniform(0, 15, (12, 3)), box, np.float64)
    group = list(range(1, 12))
    s, gr = og.nearest_distance(f, box, 0, group, beta)
    h = 1e-6
    for i in range(12):
        for a in range(3):
            fp, fm = f.copy(), f.copy()
            fp[i, a] += h
            fm[i, a] -= h
            fd = (og.nearest_distance(fp, box, 0, group, beta)[0] - og.nearest_distance(fm, box, 0, group, beta)[0]) \
                / (2 * h)
            assert abs(fd - gr.get(i, np.zeros(3))[a]) < 1e-7


def test_periodic_hill_across_the_seam():
    sig = np.array([0.35])
    c = np.array([[math.pi - 0.1]])
    V, dV = oracle.bias(np.array([-math.pi + 0.1]), c, np.array([1.2]), sig, period=[2 * math.pi])
    d = 0.2  # s - c wrapped: -2 pi + 0.2 -> +0.2
    Vexp = 1.2 * math.exp(-d * d / (2 * 0.35 ** 2))
    assert abs(V - Vexp) < 1e-14 * Vexp and abs(dV[0] - (-Vexp * d / 0.35 ** 2)) < 1e-13
    V0, _ = oracle.bias(np.array([-math.pi + 0.1]), c, np.array([1.2]), sig)
    assert V0 < 1e-30  # without the period the hill is 2 pi - 0.2 away
    # 2-D: a periodic and a non-periodic dimension
    V2, _ = oracle.bias(np.array([3.1, 0.5]), np.array([[-3.1, 0.4]]), np.array([1.0]), np.array([0.35, 0.1]),
                        period=[2 * math.pi, 0.0])
    d0 = 6.2 - 2 * math.pi
    assert abs(V2 - math.exp(-d0 * d0 / (2 * 0.35 ** 2) - 0.01 / (2 * 0.01))) < 1e-14
    # well-tempered heights see earlier hills across the seam
    kbdt = 0.0083144626 * 300.0 * 9.0
    w = oracle.deposit_sequence(np.array([[math.pi - 0.05], [-math.pi + 0.05]]), sig, 1.0, kbdt, period=[2 * math.pi])
    assert abs(w[1] - math.exp(-math.exp(-0.01 / (2 * 0.35 ** 2)) / kbdt)) < 1e-15


@pytest.mark.parametrize("kind", ["torsion", "min_dist"])
def test_step_forces_match_energy_differences(kind):
    g = np.random.default_rng(2)
    if kind == "torsion":
        box = synth.peptide_box()
        f = synth.peptide_frame(3).astype(np.float64)
        atoms, n_cv, sig, period, beta = list(synth.PEPTIDE_TORSIONS), 2, np.array([0.35, 0.35]), 2 * math.pi, 0.0
    else:
        box = np.array([15.0, 15.0, 15.0])
        f = np.zeros((30, 4))
        f[:, :3] = g.uniform(0, 15, (30, 3))
        atoms, n_cv, sig, period, beta = [0, 1] + list(range(2, 30)), 2, np.array([0.1, 0.1]), 0.0, 2.0
    s0 = np.array([r[0] for r in og.cvs(f, box, kind, atoms, n_cv, beta)])
    cen = s0 + g.normal(0.0, 1.0, (50, n_cv)) * sig
    hw = g.uniform(0.5, 1.5, 50)
    out = og.step(f, box, kind, atoms, n_cv, cen, hw, sig, beta, period=[period] * n_cv)
    assert np.abs(out["F"].sum(axis=0)).max() < 1e-9 * max(1.0, np.abs(out["F"]).max())
    h = 1e-6
    for i in sorted({int(a) for a in atoms})[:8]:
        for a in range(3):
            fp, fm = f.copy(), f.copy()
            fp[i, a] += h
            fm[i, a] -= h
            Vp = og.step(fp, box, kind, atoms, n_cv, cen, hw, sig, beta, period=[period] * n_cv)["V"]
            Vm = og.step(fm, box, kind, atoms, n_cv, cen, hw, sig, beta, period=[period] * n_cv)["V"]
            assert abs(-(Vp - Vm) / (2 * h) - out["F"][i, a]) < 1e-6 * max(1.0, np.abs(out["F"]).max())


def test_small_generators():
    box = synth.peptide_box()
    f = synth.peptide_frame(0)
    assert f.shape == (22, 4) and f.dtype == np.float32
    assert np.all((f[:, :3] >= 0) & (f[:, :3] < box))
    # backbone bonds of 1.52 A (minimum image)
    for k in range(1, synth.PEPTIDE_BACKBONE):
        d = np.array(og.displacement(f, box, k - 1, k))
        assert abs(np.linalg.norm(d) - 1.52) < 1e-4
    sw = synth.SurfaceWater()
    fr = sw.frame(0)
    assert fr.shape == (sw.n, 4) and np.all((fr[:, :3] >= 0) & (fr[:, :3] < sw.box))
    assert sw.ref not in set(sw.hydrogens.tolist()) and len(set(sw.hydrogens.tolist())) == len(sw.hydrogens)
    assert np.all(fr[sw.hydrogens, 3] == 2.0) and fr[sw.ref, 3] == 1.0


def _golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")
    out = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("="))
            out[k] = float(v)
    return out


def test_small_workloads_use_the_papers_parameters():
    """The torsion workload's hill width and height are the paper's; the
    molecule carries two four-atom torsions; the slab workload has one CV."""
    g = _golden()
    pp = synth.SMALL_PARAMS["peptide"]
    assert pp["sigma"] == (g["alanine.sigma_rad"],) * 2 and pp["w0"] == g["alanine.hill_height_kjmol"]
    assert pp["n_cv"] == g["alanine.torsions"]
    assert len(synth.PEPTIDE_TORSIONS) == g["alanine.torsions"] * g["alanine.torsion_atoms"]
    assert synth.SMALL_PARAMS["surface_water"]["n_cv"] == g["rutile.cvs"]
    assert synth.MethodParams().temperature == g["gan.temperature_k"]

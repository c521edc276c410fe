"""Pins for the oracle's box derivative (the lattice-parameter CVs of the
GaN NPT runs and the bias virial a barostat needs):
  * dV/dL_a at fixed fractional coordinates against central differences of V
    under an affine scaling of one box axis, made exact in float32 (positions
    on a 1/64 A grid, scale factors 1 +- 2^-14), with and without the
    lattice CVs, for one and two per-atom CVs;
  * the two-atom closed form: the virial of one bond along x is
    V'(s1) s'(r) r on the x axis and zero on the others.
"""
import math

import numpy as np
import pytest

import synth

oracle = pytest.importorskip("oracle")

RC = 3.5
H = 2.0 ** -14


def _grid_system(seed, n=100):
    """Atoms on a 1/64 A grid in a triaxial box, with no pair within 2e-3 A
    of rc (the switch has a kink there, which differences would straddle)."""
    box = np.array([13.5, 14.0, 15.0])  # multiples of 1/64
    g = np.random.default_rng(seed)
    for _ in range(50):
        f = g.random((n, 3))
        xyz = np.floor(f * box * 64.0) / 64.0
        d = xyz[:, None, :] - xyz[None, :, :]
        d -= box * np.round(d / box)
        r = np.sqrt((d ** 2).sum(-1))[np.triu_indices(n, 1)]
        if np.all(np.abs(r - RC) > 2e-3) and r.min() > 0.2:
            pos = np.zeros((n, 4), dtype=np.float32)
            pos[:, :3] = xyz
            pos[:, 3] = g.integers(0, 2, n)
            return pos, box
    raise RuntimeError("no clean configuration")


def _scaled(pos, box, axis, sign):
    f = 1.0 + sign * H
    p = pos.copy()
    x = pos[:, axis].astype(np.float64) * f
    assert np.array_equal(x.astype(np.float32).astype(np.float64), x)  # exact in float32
    p[:, axis] = x
    b = box.copy()
    b[axis] *= f
    return p, b


@pytest.mark.parametrize("n_cv,lattice", [(1, False), (2, False), (1, True), (2, True)])
def test_box_gradient_matches_affine_differences(n_cv, lattice):
    pos, box = _grid_system(7 + n_cv)
    D = n_cv + (3 if lattice else 0)
    sig = np.array([0.05, 0.02][:n_cv] + ([0.2, 0.2, 0.2] if lattice else []))
    p0 = oracle.make_params(box, n_cv=n_cv)
    s0 = oracle.cv(pos, p0)[0][:n_cv]
    ref = np.concatenate([s0, box]) if lattice else s0
    g = np.random.default_rng(1)
    cen = ref + g.normal(0.0, 1.5, (40, D)) * sig
    w = g.uniform(0.5, 1.5, 40)
    out = oracle.step_box(pos, p0, cen, w, sig, lattice=lattice)
    assert np.allclose(out["s"], ref, rtol=0, atol=1e-12)
    for a in range(3):
        Vs = []
        for sign in (1, -1):
            p, b = _scaled(pos, box, a, sign)
            Vs.append(oracle.step_box(p, oracle.make_params(b, n_cv=n_cv), cen, w, sig, lattice=lattice)["V"])
        fd = (Vs[0] - Vs[1]) / (2.0 * box[a] * H)
        scale = max(abs(out["box_grad"]).max(), 1e-3)
        assert abs(fd - out["box_grad"][a]) <= 1e-5 * scale, (a, fd, out["box_grad"])


def test_two_atom_virial_closed_form():
    box = np.array([10.0, 10.0, 10.0])
    r = 2.75
    pos = np.array([[3.0, 5.0, 5.0, 0.0], [3.0 + r, 5.0, 5.0, 1.0]], dtype=np.float32)
    p = oracle.make_params(box, n_cv=1)
    sig = np.array([0.05])
    c = np.array([[0.3]])
    out = oracle.step_box(pos, p, c, np.array([1.0]), sig, lattice=False)
    x, x0 = r / 2.5, 3.5 / 2.5
    sraw = lambda t: 1.0 / (1.0 + t ** 6)
    s = (sraw(x) - sraw(x0)) / (1.0 - sraw(x0))
    ds = -6.0 * x ** 5 / (2.5 * (1.0 + x ** 6) ** 2) / (1.0 - sraw(x0))
    assert abs(out["s"][0] - s) < 1e-12  # s1 = (2/N) s(r) with N = 2
    dV = -math.exp(-(s - 0.3) ** 2 / (2 * 0.05 ** 2)) * (s - 0.3) / 0.05 ** 2
    wx = dV * ds * r  # (dV/dd_x) d_x for d along x
    assert abs(out["box_grad"][0] - wx / 10.0) < 1e-12 * max(1.0, abs(wx))
    assert out["box_grad"][1] == 0.0 and out["box_grad"][2] == 0.0

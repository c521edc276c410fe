"""FP64 CPU oracle for the small-system CVs -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the baseline legs of
``bench.py`` may import this module.  The library path never does; it shares
no code with the CUDA implementation.

Two CV families of the paper's small-system runs:

* torsion angles: the alanine-dipeptide runs bias the backbone torsions
  Phi (C-N-CA-C) and Psi (N-CA-C-N), periodic angles, with sigma = 0.35 rad
  and hill height 1.2 kJ/mol (Section "Alanine dipeptide torsion", Fig. 2);
* nearest distance: the rutile runs bias the distance between one surface
  oxygen and its nearest hydrogen (Section "Water dissociation on rutile
  (110) surface", Fig. 3).

Readings where the paper is silent:

* Torsion sign: the IUPAC convention.  Looking along b -> c, the angle is
  positive when the a-b bond turns clockwise onto the c-d bond; values lie
  in [-pi, pi].  Bond vectors are minimum-image displacements.  Collinear
  atoms (an undefined angle) give 0 with a zero gradient.
* Periodic hills: a torsion is a periodic CV, so a hill sees the
  difference s - c wrapped into [-pi, pi] (the nearest image only:
  x - P * round-half-even(x / P)).
* Nearest distance: the nearest candidate is the argmin of the FP64 squared
  distance r^2 = (dx*dx + dy*dy) + dz*dz, the first in list order on a tie;
  s = sqrt(r^2).  Its gradient moves the reference atom and that candidate
  only.  The optional smooth form (beta > 0) is the soft minimum
      s = r_min - (1/beta) log sum_j exp(-beta (r_j - r_min)),
  which lies in [r_min - log(M)/beta, r_min].

Everything is plain IEEE double in Python scalars (no fused multiply-add).
Positions are float32 [N][4] frames promoted exactly to double; they are
wrapped into the box by the frame generator, so one shift of +-L gives the
minimum image.
"""
from __future__ import annotations

import math

import numpy as np


def _mi(d: float, L: float) -> float:
    if d > 0.5 * L:
        d -= L
    elif d < -0.5 * L:
        d += L
    return d


def displacement(pos4, box, i: int, j: int):
    """Minimum-image r_j - r_i (FP64)."""
    return [_mi(float(pos4[j][a]) - float(pos4[i][a]), float(box[a])) for a in range(3)]


def _dot(u, v):
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]


def _cross(u, v):
    return [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]


def _axpy(a, x, y):
    return [a * x[k] + y[k] for k in range(3)]


# ------------------------------------------------------------------ torsions

def torsion(pos4, box, quad):
    """Dihedral angle of atoms quad = (a, b, c, d), IUPAC sign, in [-pi, pi].

    Projection form: with u = r_a - r_b, e the unit vector along r_c - r_b
    and t = r_d - r_c, the components of u and t normal to e are
    v = u - (u.e) e and w = t - (t.e) e; the angle is atan2((e x v).w, v.w)."""
    a, b, c, d = (int(q) for q in quad)
    u = displacement(pos4, box, b, a)
    axis = displacement(pos4, box, b, c)
    t = displacement(pos4, box, c, d)
    ln = math.sqrt(_dot(axis, axis))
    if ln == 0.0:
        return 0.0
    e = [x / ln for x in axis]
    v = _axpy(-_dot(u, e), e, u)
    w = _axpy(-_dot(t, e), e, t)
    x = _dot(v, w)
    y = _dot(_cross(e, v), w)
    if x == 0.0 and y == 0.0:
        return 0.0
    return math.atan2(y, x)


def torsion_grad(pos4, box, quad):
    """d(phi)/d(r_a, r_b, r_c, r_d) as a 4 x 3 array.

    The classic closed form (Blondel and Karplus, J. Comput. Chem. 1996):
    with F = r_a - r_b, G = r_b - r_c, H = r_d - r_c, A = F x G, B = H x G,
        dphi/dr_a = -|G| / |A|^2 A
        dphi/dr_d = +|G| / |B|^2 B
        dphi/dr_b = |G|/|A|^2 A + (F.G)/(|A|^2 |G|) A - (H.G)/(|B|^2 |G|) B
        dphi/dr_c = -|G|/|B|^2 B - (F.G)/(|A|^2 |G|) A + (H.G)/(|B|^2 |G|) B
    Zero when the angle is undefined (A or B vanishes)."""
    a, b, c, d = (int(q) for q in quad)
    F = displacement(pos4, box, b, a)
    G = displacement(pos4, box, c, b)
    H = displacement(pos4, box, c, d)
    A = _cross(F, G)
    B = _cross(H, G)
    A2, B2 = _dot(A, A), _dot(B, B)
    g = math.sqrt(_dot(G, G))
    out = np.zeros((4, 3))
    if A2 == 0.0 or B2 == 0.0 or g == 0.0:
        return out
    fg, hg = _dot(F, G), _dot(H, G)
    for k in range(3):
        ga = -g / A2 * A[k]
        gd = g / B2 * B[k]
        out[0, k] = ga
        out[3, k] = gd
        out[1, k] = g / A2 * A[k] + fg / (A2 * g) * A[k] - hg / (B2 * g) * B[k]
        out[2, k] = -g / B2 * B[k] - fg / (A2 * g) * A[k] + hg / (B2 * g) * B[k]
    return out


# ---------------------------------------------------------- nearest distance

def _r2(dv):
    s = dv[0] * dv[0] + dv[1] * dv[1]
    return s + dv[2] * dv[2]


def nearest_distance(pos4, box, ref: int, group, beta: float = 0.0):
    """Distance from atom ref to the nearest atom of group (exact form,
    beta = 0) or its soft minimum (beta > 0).  Returns (s, grad) with grad a
    dict atom -> d s / d r_atom (3-vector)."""
    group = [int(j) for j in group]
    dvs = [displacement(pos4, box, ref, j) for j in group]
    r2 = [_r2(dv) for dv in dvs]
    m = 0
    for k in range(1, len(group)):
        if r2[k] < r2[m]:
            m = k
    rmin = math.sqrt(r2[m])
    grad = {}
    if beta <= 0.0:
        u = [x / rmin for x in dvs[m]] if rmin > 0.0 else [0.0, 0.0, 0.0]
        grad[group[m]] = np.array(u)
        grad[ref] = -np.array(u)
        return rmin, grad
    r = [math.sqrt(x) for x in r2]
    e = [math.exp(-beta * (rk - rmin)) for rk in r]
    Z = 0.0
    for x in e:
        Z += x
    s = rmin - math.log(Z) / beta
    gref = np.zeros(3)
    for k, j in enumerate(group):
        p = e[k] / Z
        u = np.array([x / r[k] for x in dvs[k]]) if r[k] > 0.0 else np.zeros(3)
        grad[j] = grad.get(j, np.zeros(3)) + p * u
        gref -= p * u
    grad[ref] = grad.get(ref, np.zeros(3)) + gref
    return s, grad


# ---------------------------------------------------------------- one step

def cvs(pos4, box, kind: str, atoms, n_cv: int, beta: float = 0.0):
    """CV values and their gradients: a list of n_cv (s_d, {atom: ds_d/dr})."""
    out = []
    if kind == "torsion":
        for d in range(n_cv):
            quad = atoms[4 * d:4 * d + 4]
            g = torsion_grad(pos4, box, quad)
            grad = {}
            for q, at in enumerate(quad):
                grad[int(at)] = grad.get(int(at), np.zeros(3)) + g[q]
            out.append((torsion(pos4, box, quad), grad))
    elif kind == "min_dist":
        group = atoms[n_cv:]
        for d in range(n_cv):
            out.append(nearest_distance(pos4, box, int(atoms[d]), group, beta))
    else:
        raise ValueError(kind)
    return out


def step(pos4, box, kind, atoms, n_cv, centres, heights, sigma, beta=0.0, period=None):
    """One frame: CVs, bias (hills, periodic differences for torsions) and
    forces F = -sum_d dV/ds_d ds_d/dr -> dict(s, V, dV, F)."""
    import oracle
    pos4 = np.asarray(pos4)
    res = cvs(pos4, box, kind, atoms, n_cv, beta)
    s = np.array([r[0] for r in res])
    V, dV = oracle.bias(s, centres, heights, sigma, period=period)
    F = np.zeros((pos4.shape[0], 3))
    for d in range(n_cv):
        for at, g in res[d][1].items():
            F[at] -= dV[d] * g
    return {"s": s, "V": V, "dV": dV, "F": F}

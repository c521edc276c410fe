"""Seeded synthetic small systems for the torsion and nearest-distance CVs.

Like ``workloads``, this module holds no arithmetic of the method (no
torsion or distance CV, no hills): it builds atom positions, atom lists and
hill centres.  Two shapes stand in for the paper's small-system runs, whose
structures and trajectories are not used:

* ``peptide``: a 22-atom chain molecule (the size of alanine dipeptide) in a
  periodic box, with two backbone torsion quadruplets sharing three atoms,
  as Phi (C-N-CA-C) and Psi (N-CA-C-N) do (Section "Alanine dipeptide
  torsion").  Each frame is an independent random conformation: backbone
  bonds of 1.52 A at bond angles drawn in [105, 120] degrees by rejection,
  13 pendant atoms 1.0-1.1 A from random backbone atoms, the whole placed
  at a random point of the box and wrapped, so bonds may cross its faces.
  The torsions then cover the whole circle.
* ``surface_water``: a rutile-like TiO2 slab (tetragonal cell a = 4.594,
  c = 2.959 A, oxygen parameter 0.305) under a layer of water molecules
  (O-H 0.96 A, H-O-H 104.5 degrees, oxygens at least 2.7 A apart), with one
  top-layer slab oxygen as the reference atom and every water hydrogen as
  a candidate (Section "Water dissociation on rutile (110) surface").
  Frame f perturbs every atom by N(0, 0.05^2) and moves one water rigidly so
  that its first hydrogen sits at a distance drawn in [0.9, 3.6] A above the
  reference oxygen, so the nearest distance spans the range of Fig. 3b.

Species ids in column 3: 0 carbon-like / titanium, 1 oxygen-like, 2 hydrogen.
"""
from __future__ import annotations

import math

import numpy as np

from .workloads import rng, wrap_to_box

PEPTIDE_CFG = 6
SURFACE_CFG = 7

PEPTIDE_ATOMS = 22
PEPTIDE_BACKBONE = 9
PEPTIDE_BOX = 24.0
# Phi and Psi as consecutive quadruplets of the backbone chain (3 atoms shared)
PEPTIDE_TORSIONS = (2, 3, 4, 5, 3, 4, 5, 6)

# Method parameters of the two small-system workloads (plain numbers; the
# torsion runs state sigma 0.35 rad and hill height 1.2 kJ/mol; the rest are
# readings: plain metadynamics for the torsions, well-tempered for the
# distance as Fig. 3 names, sigma 0.1 A).
SMALL_PARAMS = {
    "peptide": dict(n_cv=2, sigma=(0.35, 0.35), w0=1.2, biasfactor=math.inf, temperature=300.0, hills=10000,
                    period=2.0 * math.pi),
    "surface_water": dict(n_cv=1, sigma=(0.1,), w0=1.0, biasfactor=10.0, temperature=300.0, hills=1500,
                          cv_lo=0.9, cv_hi=3.6),
}


def _unit(g: np.random.Generator) -> np.ndarray:
    v = g.normal(size=3)
    return v / np.linalg.norm(v)


def peptide_frame(frame: int, sys: int = 0) -> np.ndarray:
    """One random conformation, float32 [22, 4], wrapped into the box."""
    g = rng(PEPTIDE_CFG, sys, 1, frame)
    xyz = np.zeros((PEPTIDE_ATOMS, 3))
    prev = _unit(g)
    for k in range(1, PEPTIDE_BACKBONE):
        while True:
            u = _unit(g)
            ang = math.degrees(math.acos(max(-1.0, min(1.0, float(-prev @ u)))))
            if k == 1 or 105.0 <= ang <= 120.0:
                break
        xyz[k] = xyz[k - 1] + 1.52 * u
        prev = u
    for k in range(PEPTIDE_BACKBONE, PEPTIDE_ATOMS):
        host = int(g.integers(0, PEPTIDE_BACKBONE))
        xyz[k] = xyz[host] + g.uniform(1.0, 1.1) * _unit(g)
    box = np.full(3, PEPTIDE_BOX)
    xyz += g.uniform(0.0, PEPTIDE_BOX, size=3)
    out = np.empty((PEPTIDE_ATOMS, 4), dtype=np.float32)
    out[:, :3] = wrap_to_box(xyz, box)
    species = np.full(PEPTIDE_ATOMS, 2.0, dtype=np.float32)
    species[:PEPTIDE_BACKBONE] = 0.0
    out[:, 3] = species
    return out


def peptide_box() -> np.ndarray:
    return np.full(3, PEPTIDE_BOX)


def torus_centres(sys: int, count: int, n_cv: int = 2) -> np.ndarray:
    """Hill centres uniform on [-pi, pi)^n_cv."""
    u = rng(PEPTIDE_CFG, sys, 2).random((count, n_cv))
    return -math.pi + 2.0 * math.pi * u


def interval_centres(cfg: int, sys: int, count: int, lo: float, hi: float) -> np.ndarray:
    """Hill centres uniform in [lo, hi)."""
    return lo + (hi - lo) * rng(cfg, sys, 2).random((count, 1))


RUTILE_A = 4.594
RUTILE_C = 2.959
RUTILE_U = 0.305


class SurfaceWater:
    """Slab + water system: base frame, box, reference oxygen, hydrogen list."""

    def __init__(self, cells=(4, 4, 4), water_depth: float = 10.0, vacuum: float = 12.0, sys: int = 0):
        g = rng(SURFACE_CFG, sys, 0)
        nx, ny, nz = cells
        basis_ti = [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5)]
        u = RUTILE_U
        basis_o = [(u, u, 0.0), (1 - u, 1 - u, 0.0), (0.5 + u, 0.5 - u, 0.5), (0.5 - u, 0.5 + u, 0.5)]
        cell = np.array([RUTILE_A, RUTILE_A, RUTILE_C])
        slab, sp = [], []
        for i in range(nx):
            for j in range(ny):
                for k in range(nz):
                    for b in basis_ti:
                        slab.append((np.array(b) + (i, j, k)) * cell)
                        sp.append(0.0)
                    for b in basis_o:
                        slab.append((np.array(b) + (i, j, k)) * cell)
                        sp.append(1.0)
        slab = np.array(slab)
        top = slab[:, 2].max()
        Lx, Ly = nx * RUTILE_A, ny * RUTILE_A
        z0 = top + 2.0
        Lz = z0 + water_depth + vacuum
        self.box = np.array([Lx, Ly, Lz])
        # water oxygens by rejection at density 0.033 / A^3, >= 2.7 A apart
        n_w = int(round(0.033 * Lx * Ly * water_depth))
        ow = []
        tries = 0
        while len(ow) < n_w:
            tries += 1
            if tries > 200000:
                raise RuntimeError("water placement failed")
            p = np.array([g.uniform(0, Lx), g.uniform(0, Ly), g.uniform(z0, z0 + water_depth)])
            ok = True
            for q in ow:
                d = p - q
                d[:2] -= np.round(d[:2] / self.box[:2]) * self.box[:2]
                if d @ d < 2.7 * 2.7:
                    ok = False
                    break
            if ok:
                ow.append(p)
        xyz = [*slab]
        species = list(sp)
        h_idx = []
        self.waters = []
        cos_hoh = math.cos(math.radians(104.5))
        for p in ow:
            a = _unit(g)
            t = _unit(g)
            t -= (t @ a) * a
            t /= np.linalg.norm(t)
            b = cos_hoh * a + math.sqrt(1.0 - cos_hoh * cos_hoh) * t
            io = len(xyz)
            xyz += [p, p + 0.96 * a, p + 0.96 * b]
            species += [1.0, 2.0, 2.0]
            h_idx += [io + 1, io + 2]
            self.waters.append(io)
        xyz = np.array(xyz)
        # reference: the top-layer slab oxygen nearest the middle of the face
        o_slab = [i for i in range(len(slab)) if sp[i] == 1.0 and slab[i, 2] > top - 0.5]
        mid = np.array([Lx / 2, Ly / 2])
        self.ref = int(min(o_slab, key=lambda i: float(np.sum((slab[i, :2] - mid) ** 2))))
        self.hydrogens = np.array(h_idx, dtype=np.int32)
        self.xyz = xyz
        self.species = np.array(species, dtype=np.float32)
        self.sys = sys

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def frame(self, f: int, sigma: float = 0.05) -> np.ndarray:
        g = rng(SURFACE_CFG, self.sys, 1, f)
        xyz = self.xyz + g.normal(0.0, sigma, size=self.xyz.shape)
        # move one water so that its first hydrogen lies at distance d above
        # the reference oxygen
        w = self.waters[int(g.integers(0, len(self.waters)))]
        d = g.uniform(0.9, 3.6)
        v = _unit(g)
        v[2] = abs(v[2])
        target = xyz[self.ref] + d * v
        xyz[w:w + 3] += target - xyz[w + 1]
        out = np.empty((self.n, 4), dtype=np.float32)
        out[:, :3] = wrap_to_box(xyz, self.box)
        out[:, 3] = self.species
        return out

    def cv_atoms(self) -> np.ndarray:
        """Reference atom first, then the candidate group."""
        return np.concatenate([[self.ref], self.hydrogens]).astype(np.int32)

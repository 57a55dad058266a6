"""Seeded synthetic workloads for RHEED/TRHEPD rocking-curve simulations.

This module only *describes inputs*: lattice vectors, the integer beam list, atom positions,
Debye-Waller factors, scattering-factor parameters, energy and glancing angles. It holds none of
the arithmetic of the simulation method (no wavenumbers, no potential, no integrator), so both the
CUDA path and the CPU oracle can consume the same inputs without sharing any of the method.

The problem statement it feeds is the paper's Section 2.1: a 2D-periodic surface slab
(lattice a1, a2), beams k_j = m1*b1 + m2*b2 with k_1 = 0, incident altitude theta0 and azimuth
theta1, bottom boundary z_e < 0 and L slices of width h = -z_e / L.

Recipes (all seeds go through ``numpy.random.default_rng``):

* ``rheed_row`` (one angle, 11 beams): 15 keV electrons, square 3.8 A cell, beams m*b1 for
  m = -5..5 ordered 0, +1, -1, ..., 8 layers x 2 atoms at z = -3.35 - 1.9 k +- U(0.1) A,
  in-plane positions uniform in the cell, B = 0.5 A^2, absorption 0.1, 20 A slab in 400 slices,
  theta0 = 2.0 deg, theta1 = 90 deg (incidence perpendicular to the beam row).
* ``trhepd_n61`` (rocking curve, 61 beams): 10 keV positrons, hexagonal 3.84 A cell, beams with
  |g|^2 <= 16 |b*|^2, 6 surface atoms with z ~ U[-4.5, -3.0] over 10 bulk atoms at
  z = -5.5 - 2.4 k, 30 A slab in 2000 slices of 0.015 A, theta0 = 0.5..6.4 deg in 0.1 deg steps,
  theta1 = 0.
* ``batch_sets``: perturbations of the 61-beam structure's surface z by N(0, 0.3^2) A, beam
  counts cycling through 31 / 61 / 121 (hexagonal shells |g|^2/|b*|^2 <= 7 / 16 / 31).
* ``rfactor_fit``: 12 free surface atoms in 6 Debye-Waller classes over a 10-layer bulk, hidden
  true parameters and a perturbed starting point.
* ``large_n255``: square 5.4 A cell, 255 beams (smallest |g| with tie-break |g|^2, m1, m2),
  8 surface atoms over the same bulk, 3000 slices of 0.01 A, 120 angles in 0.2..6.2 deg.

Structure seeds are 1000 + recipe index, scattering-factor seeds 2000 + recipe index.
Scattering factors are 4 Gaussians per species, a_i ~ U[0.1, 2] A and b_i ~ U[0.5, 50] A^2.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import List

import numpy as np


@dataclass
class Workload:
    name: str
    particle: int            # +1 electron (RHEED), -1 positron (TRHEPD)
    energy_ev: float         # kinetic energy (eV)
    absorption: float        # absorptive potential as a fraction of the real potential
    a1: np.ndarray           # (2,) surface lattice vector (A)
    a2: np.ndarray           # (2,) surface lattice vector (A)
    beams: np.ndarray        # (N, 2) int32 beam indices (m1, m2); beams[0] == (0, 0)
    atoms: np.ndarray        # (n_atoms, 3) x, y, z in A (z <= 0: inside the slab)
    dw: np.ndarray           # (n_atoms,) Debye-Waller B factor (A^2)
    species: np.ndarray      # (n_atoms,) int32 species index
    sf: np.ndarray           # (n_species, 8) scattering factor a_1..a_4 (A), b_1..b_4 (A^2)
    z_e: float               # slab bottom (A), < 0
    n_steps: int             # number of slices L; h = -z_e / L
    theta0: np.ndarray       # (A,) glancing angles (degrees)
    theta1: np.ndarray       # (A,) azimuths measured from a1 (degrees)

    @property
    def n_beams(self) -> int:
        return int(self.beams.shape[0])

    @property
    def h(self) -> float:
        return -self.z_e / self.n_steps

    def with_angles(self, theta0, theta1=None) -> "Workload":
        theta0 = np.atleast_1d(np.asarray(theta0, dtype=np.float64))
        if theta1 is None:
            theta1 = np.full_like(theta0, float(self.theta1[0]))
        return replace(self, theta0=theta0,
                       theta1=np.atleast_1d(np.asarray(theta1, dtype=np.float64)))

    def with_steps(self, n_steps: int) -> "Workload":
        return replace(self, n_steps=int(n_steps))


# ----------------------------------------------------------------------------------------------
# lattices and integer beam lists
# ----------------------------------------------------------------------------------------------

def square_lattice(a: float):
    return np.array([a, 0.0]), np.array([0.0, a])


def hex_lattice(a: float):
    return np.array([a, 0.0]), np.array([0.5 * a, 0.5 * np.sqrt(3.0) * a])


def beam_row(m_max: int) -> np.ndarray:
    """Beams m*b1 for m = 0, +1, -1, +2, -2, ..., +m_max, -m_max."""
    out = [(0, 0)]
    for m in range(1, m_max + 1):
        out += [(m, 0), (-m, 0)]
    return np.array(out, dtype=np.int32)


def _reciprocal_gram(a1, a2):
    # Gram matrix of the reciprocal basis (only used to rank beams by length).
    A = np.array([a1, a2], dtype=np.float64)
    B = 2.0 * np.pi * np.linalg.inv(A).T
    return B @ B.T


def beam_disk(a1, a2, n_beams: int, m_range: int = 40) -> np.ndarray:
    """The n_beams shortest reciprocal-lattice rods, (0,0) first, ties broken by (m1, m2)."""
    G = _reciprocal_gram(a1, a2)
    m = np.arange(-m_range, m_range + 1)
    m1, m2 = [x.ravel() for x in np.meshgrid(m, m, indexing="ij")]
    q = G[0, 0] * m1 * m1 + 2 * G[0, 1] * m1 * m2 + G[1, 1] * m2 * m2
    q = np.round(q / G[0, 0], 9)
    order = np.lexsort((m2, m1, q))
    sel = order[:n_beams]
    return np.stack([m1[sel], m2[sel]], axis=1).astype(np.int32)


def beam_shell(a1, a2, radius2_in_b: float) -> np.ndarray:
    """All rods with |g|^2 <= radius2_in_b * |b1|^2, (0,0) first, ordered by (|g|^2, m1, m2)."""
    G = _reciprocal_gram(a1, a2)
    m = np.arange(-40, 41)
    m1, m2 = [x.ravel() for x in np.meshgrid(m, m, indexing="ij")]
    q = G[0, 0] * m1 * m1 + 2 * G[0, 1] * m1 * m2 + G[1, 1] * m2 * m2
    q = np.round(q / G[0, 0], 9)
    keep = q <= radius2_in_b + 1e-9
    m1, m2, q = m1[keep], m2[keep], q[keep]
    order = np.lexsort((m2, m1, q))
    return np.stack([m1[order], m2[order]], axis=1).astype(np.int32)


# ----------------------------------------------------------------------------------------------
# structures
# ----------------------------------------------------------------------------------------------

def scattering_factors(seed: int, n_species: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.1, 2.0, size=(n_species, 4))
    b = rng.uniform(0.5, 50.0, size=(n_species, 4))
    return np.concatenate([a, b], axis=1)


def _inplane(rng, a1, a2, n):
    f = rng.uniform(0.0, 1.0, size=(n, 2))
    return f[:, :1] * a1[None, :] + f[:, 1:] * a2[None, :]


def rheed_row() -> Workload:
    """15 keV electrons, 11-beam row, 16 atoms in 8 layers, one glancing angle (2.0 deg)."""
    rng = np.random.default_rng(1000)
    a1, a2 = square_lattice(3.8)
    n_layers, per_layer = 8, 2
    z = []
    for k in range(n_layers):
        for _ in range(per_layer):
            z.append(-3.35 - 1.9 * k + rng.uniform(-0.1, 0.1))
    xy = _inplane(rng, a1, a2, n_layers * per_layer)
    atoms = np.concatenate([xy, np.array(z)[:, None]], axis=1)
    n = atoms.shape[0]
    return Workload(
        name="rheed_row_n11", particle=+1, energy_ev=15000.0, absorption=0.1,
        a1=a1, a2=a2, beams=beam_row(5), atoms=atoms, dw=np.full(n, 0.5),
        species=np.zeros(n, dtype=np.int32), sf=scattering_factors(2000),
        z_e=-20.0, n_steps=400, theta0=np.array([2.0]), theta1=np.array([90.0]))


def _trhepd_bulk(rng, a1, a2, z_top=-5.5, dz=2.4, n_layers=10):
    z = z_top - dz * np.arange(n_layers)
    xy = _inplane(rng, a1, a2, n_layers)
    return np.concatenate([xy, z[:, None]], axis=1)


def trhepd_n61() -> Workload:
    """10 keV positrons, 61 beams, 6 surface atoms + 10 bulk layers, 60 glancing angles."""
    rng = np.random.default_rng(1001)
    a1, a2 = hex_lattice(3.84)
    surf_xy = _inplane(rng, a1, a2, 6)
    surf_z = rng.uniform(-4.5, -3.0, size=6)
    surf = np.concatenate([surf_xy, surf_z[:, None]], axis=1)
    bulk = _trhepd_bulk(rng, a1, a2)
    atoms = np.concatenate([surf, bulk], axis=0)
    n = atoms.shape[0]
    theta0 = np.round(0.5 + 0.1 * np.arange(60), 10)
    return Workload(
        name="trhepd_n61", particle=-1, energy_ev=10000.0, absorption=0.1,
        a1=a1, a2=a2, beams=beam_shell(a1, a2, 16.0), atoms=atoms, dw=np.full(n, 0.5),
        species=np.zeros(n, dtype=np.int32), sf=scattering_factors(2001),
        z_e=-30.0, n_steps=2000, theta0=theta0, theta1=np.zeros(60))


N_SURFACE_61 = 6  # the first 6 atoms of trhepd_n61() are the surface atoms


def batch_sets(n_sets: int = 512, beam_classes=(31, 61, 121)) -> List[Workload]:
    """Parameter sets: surface z of ``trhepd_n61`` perturbed by N(0, 0.3^2) A (seed 3000 + k);
    set k uses the hexagonal shell with beam_classes[k % len(beam_classes)] beams."""
    base = trhepd_n61()
    radius = {31: 7.0, 61: 16.0, 121: 31.0}
    out = []
    for k in range(n_sets):
        rng = np.random.default_rng(3000 + k)
        atoms = base.atoms.copy()
        atoms[:N_SURFACE_61, 2] += rng.normal(0.0, 0.3, size=N_SURFACE_61)
        atoms[:, 2] = np.minimum(atoms[:, 2], -0.5)
        nb = beam_classes[k % len(beam_classes)]
        beams = beam_shell(base.a1, base.a2, radius[nb])
        assert beams.shape[0] == nb
        out.append(replace(base, name=f"set{k}_n{nb}", atoms=atoms, beams=beams))
    return out


@dataclass
class FitProblem:
    """R-factor fit: 12 free surface z coordinates and 6 Debye-Waller classes (2 atoms each)."""
    workload: Workload          # structure at the starting point
    free_atoms: np.ndarray      # (12,) indices of atoms whose z is a parameter
    dw_class: np.ndarray        # (n_atoms,) class index 0..5 for free atoms, -1 otherwise
    z_true: np.ndarray          # (12,)
    b_true: np.ndarray          # (6,)
    z_start: np.ndarray         # (12,)
    b_start: np.ndarray         # (6,)


def rfactor_fit() -> FitProblem:
    rng = np.random.default_rng(1003)
    a1, a2 = hex_lattice(3.84)
    n_free = 12
    xy = _inplane(rng, a1, a2, n_free)
    z0 = np.concatenate([rng.uniform(-3.5, -2.5, 6), rng.uniform(-5.0, -4.0, 6)])
    bulk = _trhepd_bulk(rng, a1, a2, z_top=-6.5, dz=2.35)
    rt = np.random.default_rng(4000)
    z_true = z0 + rt.normal(0.0, 0.1, n_free)
    b_true = 0.5 + rt.uniform(-0.2, 0.2, 6)
    rs = np.random.default_rng(4001)
    z_start = z_true + rs.normal(0.0, 0.05, n_free)
    b_start = b_true + rs.normal(0.0, 0.05, 6)
    atoms = np.concatenate([np.concatenate([xy, z_start[:, None]], axis=1), bulk], axis=0)
    n = atoms.shape[0]
    dw_class = -np.ones(n, dtype=np.int32)
    dw_class[:n_free] = np.arange(n_free) // 2
    dw = np.full(n, 0.5)
    dw[:n_free] = b_start[dw_class[:n_free]]
    theta0 = np.round(0.5 + 0.1 * np.arange(60), 10)
    wl = Workload(
        name="rfactor_fit_n61", particle=-1, energy_ev=10000.0, absorption=0.1,
        a1=a1, a2=a2, beams=beam_shell(a1, a2, 16.0), atoms=atoms, dw=dw,
        species=np.zeros(n, dtype=np.int32), sf=scattering_factors(2003),
        z_e=-30.0, n_steps=2000, theta0=theta0, theta1=np.zeros(60))
    return FitProblem(wl, np.arange(n_free), dw_class, z_true, b_true, z_start, b_start)


def fit_structure(fp: FitProblem, z: np.ndarray, b: np.ndarray) -> Workload:
    """The fit workload with free z coordinates ``z`` (12,) and class B factors ``b`` (6,)."""
    atoms = fp.workload.atoms.copy()
    atoms[fp.free_atoms, 2] = z
    dw = fp.workload.dw.copy()
    m = fp.dw_class >= 0
    dw[m] = np.asarray(b)[fp.dw_class[m]]
    return replace(fp.workload, atoms=atoms, dw=dw)


def large_n255(n_sets: int = 64) -> List[Workload]:
    rng = np.random.default_rng(1004)
    a1, a2 = square_lattice(5.4)
    surf_xy = _inplane(rng, a1, a2, 8)
    surf_z = rng.uniform(-4.5, -3.0, size=8)
    bulk = _trhepd_bulk(rng, a1, a2)
    base_atoms = np.concatenate([np.concatenate([surf_xy, surf_z[:, None]], axis=1), bulk])
    n = base_atoms.shape[0]
    beams = beam_disk(a1, a2, 255)
    theta0 = np.linspace(0.2, 6.2, 120)
    out = []
    for k in range(n_sets):
        r = np.random.default_rng(5000 + k)
        atoms = base_atoms.copy()
        atoms[:8, 2] += r.normal(0.0, 0.3, 8)
        atoms[:, 2] = np.minimum(atoms[:, 2], -0.5)
        out.append(Workload(
            name=f"large_set{k}_n255", particle=-1, energy_ev=10000.0, absorption=0.1,
            a1=a1, a2=a2, beams=beams, atoms=atoms, dw=np.full(n, 0.5),
            species=np.zeros(n, dtype=np.int32), sf=scattering_factors(2004),
            z_e=-30.0, n_steps=3000, theta0=theta0, theta1=np.zeros(120)))
    return out


def tiny(n_beams: int = 3, n_steps: int = 20, seed: int = 7, particle: int = -1,
         absorption: float = 0.1, theta0=(1.5,), energy_ev: float = 10000.0,
         depth: float = 6.0) -> Workload:
    """Small random problems for brute-force and order tests (hexagonal 3.84 A cell)."""
    rng = np.random.default_rng(seed)
    a1, a2 = hex_lattice(3.84)
    beams = beam_disk(a1, a2, n_beams)
    n_atoms = 4
    xy = _inplane(rng, a1, a2, n_atoms)
    z = rng.uniform(-depth + 1.0, -1.0, size=n_atoms)
    atoms = np.concatenate([xy, z[:, None]], axis=1)
    theta0 = np.atleast_1d(np.asarray(theta0, dtype=np.float64))
    return Workload(
        name=f"tiny_n{n_beams}", particle=particle, energy_ev=energy_ev, absorption=absorption,
        a1=a1, a2=a2, beams=beams, atoms=atoms, dw=np.full(n_atoms, 0.5),
        species=np.zeros(n_atoms, dtype=np.int32), sf=scattering_factors(seed + 100),
        z_e=-depth, n_steps=n_steps, theta0=theta0, theta1=np.zeros_like(theta0))


RECIPES = {
    "rheed_row_n11": rheed_row,
    "trhepd_n61": trhepd_n61,
}

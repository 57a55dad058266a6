"""Oracle for the bulk layer: the converged bulk boundary condition below the surface slab.

TEST INFRASTRUCTURE (see ``oracle/model.py``): not used by the CUDA path.

Below z_e the crystal is an ideal bulk, periodic in z with period d. The paper (Section 2.2, end)
computes the bulk's reflection once, stops when it has converged and reuses it for every
structure of the search. In the economical form of Algorithm 1 the same information is the
normalised state X = P Q^{-1} at z_e of the solutions that belong in the bulk (a matrix of
logarithmic derivatives: c' = X c). One bulk period maps X at its bottom to X at its top:

    F(X): integrate Z from [I; X] over one period with Algorithm 1's step, then X' = P Q^{-1},

and the semi-infinite bulk's X is the fixed point X = F(X). Iterating from the no-wave value
X_0 = i Gamma (rho = 0 at the bottom of a deep bulk) adds one period below per iteration; the
iteration stops when the largest entry of X changes by less than ``tol`` times the largest
entry. The slab is then integrated from [I; X_bulk] instead of [I; i Gamma].

``bulk_potential`` builds the periodic bulk potential from the atoms of one period (z relative
to the period top, in (-d, 0]) and their images, with the model of ``oracle/model.py``.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from .integrator import integrate, splitting_coefficients  # noqa: F401  (scheme names)
from .model import Angle, Potential


def bulk_images(atoms_rel, dw, species, z_top: float, period: float, reach: float = 8.0):
    """Atoms of the periodic bulk around one period [z_top - d, z_top]: the period's atoms
    shifted by z_top + k d for every k with |k d| <= reach + d (Gaussian tails beyond ~7 A are
    below 1e-16 for B <= 50 A^2)."""
    atoms_rel = np.asarray(atoms_rel, dtype=np.float64)
    kmax = int(np.ceil((reach + period) / period))
    out, dws, sps = [], [], []
    for k in range(-kmax, kmax + 1):
        a = atoms_rel.copy()
        a[:, 2] = a[:, 2] + z_top + k * period
        out.append(a)
        dws.append(np.asarray(dw, dtype=np.float64))
        sps.append(np.asarray(species))
    return np.concatenate(out), np.concatenate(dws), np.concatenate(sps)


def bulk_potential(wl, atoms_rel, dw, species, period: float) -> Potential:
    """U(z) of the ideal bulk with the beams, lattice and scattering factors of ``wl``."""
    at, d, sp = bulk_images(atoms_rel, dw, species, wl.z_e, period)
    return Potential(replace(wl, atoms=at, dw=d, species=sp))


def period_map(Gam, gam2, Ufun, X, z_bottom: float, period: float, steps: int, scheme: str,
               threshold: float = 1000.0):
    """F(X): one period of Algorithm 1's integration from [I; X] at z_bottom, normalised."""
    n = len(Gam)
    Z0 = np.vstack([np.eye(n, dtype=np.complex128), np.asarray(X, dtype=np.complex128)])
    Q, P, _ = integrate(Gam, gam2, Ufun, z_bottom, steps, scheme, threshold, Z0=Z0,
                        span=period)
    return np.linalg.solve(Q.T, P.T).T


def bulk_x(Gam, gam2, Ufun, z_top: float, period: float, steps: int, scheme: str = "sp4",
           tol: float = 1e-12, max_periods: int = 500, threshold: float = 1000.0):
    """The fixed point X_bulk of the period map, iterated from X = i Gamma; returns
    (X_bulk, periods used, last relative change)."""
    X = np.diag(1j * np.asarray(Gam))
    change = np.inf
    for k in range(1, max_periods + 1):
        Xn = period_map(Gam, gam2, Ufun, X, z_top - period, period, steps, scheme, threshold)
        change = np.max(np.abs(Xn - X)) / np.max(np.abs(Xn))
        X = Xn
        if change < tol:
            return X, k, change
    return X, max_periods, change


def rho_with_bulk(Gam, gam2, Ufun, X_bulk, z_e: float, L: int, scheme: str = "sp4",
                  threshold: float = 1000.0):
    """rho(0) of the slab integrated from [I; X_bulk] at z_e (Eq. vrhocomp times Q)."""
    from .integrator import assemble
    n = len(Gam)
    Z0 = np.vstack([np.eye(n, dtype=np.complex128), np.asarray(X_bulk, dtype=np.complex128)])
    Q, P, n_rhst = integrate(Gam, gam2, Ufun, z_e, L, scheme, threshold, Z0=Z0)
    return assemble(Gam, Q, P), n_rhst


def angle_bulk(wl, bulk_atoms, bulk_dw, bulk_species, period: float, steps: int,
               theta0: float, theta1: float, scheme: str = "sp4", tol: float = 1e-12):
    """(X_bulk, periods, rho, eta) for one direction of a workload over an ideal bulk."""
    from .model import intensities
    ang = Angle(wl, theta0, theta1)
    bpot = bulk_potential(wl, bulk_atoms, bulk_dw, bulk_species, period)
    X, k, _ = bulk_x(ang.Gam, ang.gam2, bpot.U, wl.z_e, period, steps, scheme, tol)
    pot = Potential(wl)
    rho, _ = rho_with_bulk(ang.Gam, ang.gam2, pot.U, X, wl.z_e, wl.n_steps, scheme)
    eta, _ = intensities(rho, ang.gam2, theta0)
    return X, k, rho, eta

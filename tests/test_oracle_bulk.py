"""Pins for the bulk-layer oracle (oracle/bulk.py): closed forms for a uniform bulk, the fixed
point of the period map, and agreement with an explicit deep integration."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import bulk as B
from oracle.closed_forms import half_space_rho
from oracle.integrator import integrate, assemble
from oracle.model import Angle, Potential
from paper_2306_00271_gb300 import workloads as W


def _one_beam(U0=4.0 - 0.4j, G=0.35):
    return np.array([G], dtype=np.complex128), np.array([G * G]), (lambda z: np.array([[U0]]))


def test_uniform_bulk_is_the_decaying_mode():
    """One beam in a uniform absorbing bulk: c'' = -K^2 c, the bulk solution is exp(iKz) with
    Im K <= 0 (decaying into the bulk), so X = c'/c = iK."""
    Gam, gam2, U = _one_beam()
    K = np.sqrt(gam2[0] + U(0)[0, 0])
    K = K if K.imag <= 0 else -K
    X, k, change = B.bulk_x(Gam, gam2, U, z_top=-5.0, period=2.0, steps=80, tol=1e-13)
    assert change < 1e-13 and k > 3
    assert abs(X[0, 0] - 1j * K) < 1e-9 * abs(K)


def test_half_space_closed_form():
    """A uniform potential below z = 0 (bulk and slab alike): rho is the half-space Fresnel
    coefficient (Gamma - K) / (Gamma + K)."""
    U0, G = 4.0 - 0.4j, 0.35
    Gam, gam2, U = _one_beam(U0, G)
    X, _, _ = B.bulk_x(Gam, gam2, U, z_top=-3.0, period=1.5, steps=120, tol=1e-14)
    rho, _ = B.rho_with_bulk(Gam, gam2, U, X, z_e=-3.0, L=240)
    assert abs(rho[0] - half_space_rho(G, U0)) < 1e-9


def _bulk_case():
    # strong absorption: the bulk memory of the deep start fades by ~e^-1 per period, so the
    # iteration converges in tens of periods (weakly absorbing bulks need hundreds)
    wl = W.tiny(n_beams=3, seed=5, n_steps=40, theta0=(1.3,), depth=4.8, absorption=0.6)
    bulk_atoms = np.array([[0.7, 0.4, -1.1], [2.1, 1.5, -2.0]])
    return wl, bulk_atoms, np.array([0.5, 0.7]), np.zeros(2, dtype=np.int32), 2.4


def test_period_map_fixed_point():
    wl, atoms, dw, sp, d = _bulk_case()
    ang = Angle(wl, wl.theta0[0], wl.theta1[0])
    pot = B.bulk_potential(wl, atoms, dw, sp, d)
    X, k, change = B.bulk_x(ang.Gam, ang.gam2, pot.U, wl.z_e, d, 48, tol=1e-12)
    assert change < 1e-12
    Xn = B.period_map(ang.Gam, ang.gam2, pot.U, X, wl.z_e - d, d, 48, "sp4")
    assert np.max(np.abs(Xn - X)) < 1e-11 * np.max(np.abs(X))


def test_bulk_condition_equals_deep_explicit_integration():
    """Slab made of two bulk periods on top of the ideal bulk: starting the slab from X_bulk
    gives the same rho as integrating the periodic potential explicitly from 120 periods deep
    with the no-wave start (the deep start's influence has decayed)."""
    wl, atoms, dw, sp, d = _bulk_case()
    wl = replace(wl, z_e=-2 * d, n_steps=96)
    ang = Angle(wl, wl.theta0[0], wl.theta1[0])
    K = 120
    at, dws, sps = B.bulk_images(atoms, dw, sp, 0.0, d, reach=(K + 4) * d)
    deep = Potential(replace(wl, atoms=at, dw=dws, species=sps))
    X, k, _ = B.bulk_x(ang.Gam, ang.gam2, deep.U, wl.z_e, d, 48, tol=1e-13)
    assert k < K
    rho_b, _ = B.rho_with_bulk(ang.Gam, ang.gam2, deep.U, X, wl.z_e, wl.n_steps)
    Q, P, _ = integrate(ang.Gam, ang.gam2, deep.U, wl.z_e - K * d, wl.n_steps + 48 * K, "sp4",
                        1000.0)
    rho_e = assemble(ang.Gam, Q, P)
    assert np.max(np.abs(rho_b - rho_e)) < 1e-10 * np.max(np.abs(rho_e))

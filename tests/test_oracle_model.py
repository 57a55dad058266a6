"""Pins of the oracle's physics model (Section 2.1) against definitions it does not reuse."""
import numpy as np
import pytest

from oracle import model
from paper_2306_00271_gb300 import workloads as W


def test_prefactor_is_textbook_constant():
    # u_g [1/A^2] = (2 m gamma_L e / hbar^2) V_g and V_g = (h^2 / (2 pi m e Omega)) F_g with the
    # textbook 47.878 V*A^2; their product must be 4 pi gamma_L / Omega.
    volt_a2 = 47.878
    per_ev = 2.0 * model.MC2_EV / model.HBARC_EV_A ** 2
    assert abs(volt_a2 * per_ev - 4 * np.pi) / (4 * np.pi) < 2e-4


def test_wavenumber_10kev():
    # lambda(10 keV, relativistic) = 0.12204 A (textbook), gamma = 2 pi / lambda.
    g = model.vacuum_wavenumber(10000.0)
    assert abs(2 * np.pi / g - 0.12204) < 2e-5


def test_beam_shells_hexagonal_counts():
    a1, a2 = W.hex_lattice(3.84)
    for r2, n in [(7.0, 31), (16.0, 61), (31.0, 121)]:
        b = W.beam_shell(a1, a2, r2)
        assert b.shape[0] == n
        assert tuple(b[0]) == (0, 0)
        k = model.rods(b, a1, a2)
        bstar2 = np.sum(model.reciprocal_basis(a1, a2)[0] ** 2)
        assert np.all(np.sum(k * k, axis=1) <= r2 * bstar2 * (1 + 1e-12))
    row = W.beam_row(5)
    assert [tuple(x) for x in row[:5]] == [(0, 0), (1, 0), (-1, 0), (2, 0), (-2, 0)]


def test_reciprocal_basis():
    a1, a2 = W.hex_lattice(3.84)
    B = model.reciprocal_basis(a1, a2)
    A = np.array([a1, a2])
    assert np.allclose(A @ B.T, 2 * np.pi * np.eye(2), atol=1e-13)


def test_gamma_branch_and_square():
    wl = W.trhepd_n61()
    ang = model.Angle(wl, 2.0, 0.0)
    assert np.allclose(ang.Gam ** 2, ang.gam2, rtol=1e-13, atol=1e-10)
    assert np.all(ang.Gam.imag <= 0)
    assert np.all(ang.Gam.real >= 0)
    # specular beam: Gamma_1 = gamma sin(theta0)
    assert abs(ang.Gam[0] - ang.gamma * np.sin(np.deg2rad(2.0))) < 1e-12


def _real_space_potential(pot, wl, xy, z):
    """v(r) summed over atoms and lattice images: the inverse transform of the model written as
    normalised 3D Gaussians (Poisson summation of the 2D Fourier series)."""
    a1, a2 = np.asarray(wl.a1), np.asarray(wl.a2)
    C = (wl.particle - 1j * wl.absorption) * 4 * np.pi * model.lorentz_factor(wl.energy_ev)
    v = np.zeros(xy.shape[0], dtype=np.complex128)
    sf = wl.sf[wl.species]
    for at, s, B in zip(wl.atoms, sf, wl.dw):
        for i in range(4):
            beta = (s[4 + i] + B) / (16 * np.pi ** 2)
            for p in range(-3, 4):
                for q in range(-3, 4):
                    c = at[:2] + p * a1 + q * a2
                    r2 = np.sum((xy - c) ** 2, axis=1) + (z - at[2]) ** 2
                    v += C * s[i] * np.exp(-r2 / (4 * beta)) / (4 * np.pi * beta) ** 1.5
    return v


def test_potential_matches_real_space_fourier_transform():
    wl = W.tiny(n_beams=7, seed=3)
    pot = model.Potential(wl)
    a1, a2 = np.asarray(wl.a1), np.asarray(wl.a2)
    n = 96
    f = (np.arange(n) + 0.5) / n
    f1, f2 = [x.ravel() for x in np.meshgrid(f, f, indexing="ij")]
    xy = f1[:, None] * a1 + f2[:, None] * a2
    for z in (-1.3, -2.7):
        v = _real_space_potential(pot, wl, xy, z)
        # u_g = (1/A) int_cell v exp(-i g.r) d^2r  (rectangle rule: spectral for periodic v)
        u_ft = np.array([np.mean(v * np.exp(-1j * xy @ g)) for g in pot.g])
        u = pot.u(z)[0]
        assert np.max(np.abs(u_ft - u)) < 1e-9 * np.max(np.abs(u))


def test_potential_z_integral_is_scattering_factor():
    # int u_g(z) dz = (C/A) sum_a exp(-i g.r_a) f(s) exp(-B s^2), s = |g| / (4 pi).
    wl = W.tiny(n_beams=7, seed=5, depth=30.0)
    pot = model.Potential(wl)
    z = np.linspace(-60.0, 30.0, 20001)
    u = pot.u(z)
    integral = np.trapezoid(u, z, axis=0)
    C = (wl.particle - 1j * wl.absorption) * 4 * np.pi * model.lorentz_factor(wl.energy_ev)
    s = np.sqrt(pot.g2) / (4 * np.pi)
    ref = np.zeros(pot.g.shape[0], dtype=np.complex128)
    for at, sp, B in zip(wl.atoms, wl.sf[wl.species], wl.dw):
        f = sum(sp[i] * np.exp(-sp[4 + i] * s ** 2) for i in range(4))
        ref += np.exp(-1j * pot.g @ at[:2]) * f * np.exp(-B * s ** 2)
    ref *= C / pot.area
    assert np.max(np.abs(integral - ref)) < 1e-9 * np.max(np.abs(ref))


def test_index_map_is_convolution():
    # (v psi) at rod k_j must equal (U c)_j for psi = sum_k c_k exp(i k_k . r) (Eq. sch2).
    wl = W.tiny(n_beams=7, seed=11)
    pot = model.Potential(wl)
    a1, a2 = np.asarray(wl.a1), np.asarray(wl.a2)
    k = model.rods(wl.beams, a1, a2)
    rng = np.random.default_rng(0)
    c = rng.normal(size=7) + 1j * rng.normal(size=7)
    z = -2.0
    n = 64
    f = np.arange(n) / n
    f1, f2 = [x.ravel() for x in np.meshgrid(f, f, indexing="ij")]
    xy = f1[:, None] * a1 + f2[:, None] * a2
    # v(r) from its own Fourier series over all differences the beam set needs
    v = np.exp(1j * xy @ pot.g.T) @ pot.u(z)[0]
    psi = np.exp(1j * xy @ k.T) @ c
    vpsi = np.array([np.mean(v * psi * np.exp(-1j * xy @ kj)) for kj in k])
    assert np.max(np.abs(vpsi - pot.U(z) @ c)) < 1e-10 * np.max(np.abs(vpsi))


def test_absorption_sign():
    # Absorption needs Im U < 0 in the paper's convention for both particles; Re u_0 has the
    # particle's sign (attractive for electrons).
    for particle in (+1, -1):
        wl = W.tiny(n_beams=3, particle=particle)
        pot = model.Potential(wl)
        i0 = int(np.where((pot.diffs == 0).all(axis=1))[0][0])
        u0 = pot.u(np.linspace(wl.z_e, 0, 50))[:, i0]
        assert np.all(u0.imag <= 0)
        assert np.all(np.sign(u0.real[np.abs(u0.real) > 1e-12]) == particle)


def test_eta_definition():
    gam2 = np.array([4.0, 1.0, -2.0])
    rho = np.array([0.5, 0.2, 0.9])
    eta, flux = model.intensities(rho, gam2, 3.0)
    s = np.sin(np.deg2rad(3.0))
    assert np.allclose(eta, [0.25 * s, 0.04 * s * 2.0, 0.0])
    assert np.allclose(flux * s, eta)

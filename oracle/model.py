"""Oracle: physics model of the RHEED/TRHEPD boundary-value problem (plain NumPy, FP64).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA path never does.

What is computed here follows Section 2.1 of the paper (Eqs. sch1-sch3, vtau, vrho, bd0, bd1,
and the intensity formula below Eq. bd1):

* gamma = vacuum wavenumber; b0 = projection of the incident wavevector on the surface;
* Gamma = diag(sqrt(gamma^2 - |b0 + k_j|^2)) (Eq. sch3), evanescent branch Im Gamma <= 0;
* U_{jk}(z) = u_{g_j - g_k}(z) (Eq. sch2's index map l(j, k));
* eta_i = |rho_i|^2 sin(theta0) Gamma_1 / Gamma_i for propagating beams, 0 otherwise.

The paper does not state a potential model. The one used here (a reading, listed with the other
readings in the design notes) is the standard electron-scattering-factor model: per species
f(s) = sum_i a_i exp(-b_i s^2), s = |q| / (4 pi), a Debye-Waller factor B per atom, and an
absorptive part equal to a fixed fraction of the real potential with the sign that absorbs in
the paper's convention (incident wave exp(i Gamma z) travelling towards -z):

  u_g(z) = (s_p - i*absorption) * (4 pi gamma_L / A_cell)
           * sum_atoms exp(-i g.r_a) sum_i a_i exp(-beta |g|^2) exp(-(z - z_a)^2 / (4 beta)) / (2 sqrt(pi beta)),
  beta = (b_i + B_a) / (16 pi^2),

with s_p = +1 for electrons and -1 for positrons, and gamma_L = 1 + E / (m c^2).
"""
from __future__ import annotations

import numpy as np

HBARC_EV_A = 1973.269804        # hbar*c in eV*Angstrom
MC2_EV = 510998.95              # electron rest energy in eV


def vacuum_wavenumber(energy_ev: float) -> float:
    """Relativistic vacuum wavenumber gamma (1/A) of an electron/positron of kinetic energy E."""
    E = float(energy_ev)
    return np.sqrt(E * E + 2.0 * E * MC2_EV) / HBARC_EV_A


def lorentz_factor(energy_ev: float) -> float:
    return 1.0 + float(energy_ev) / MC2_EV


def reciprocal_basis(a1, a2) -> np.ndarray:
    """Rows b1, b2 with a_i . b_j = 2 pi delta_ij."""
    A = np.array([a1, a2], dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(A).T


def rods(beams, a1, a2) -> np.ndarray:
    """Reciprocal rods k_j = m1 b1 + m2 b2 (N, 2) in 1/A."""
    B = reciprocal_basis(a1, a2)
    return np.asarray(beams, dtype=np.float64) @ B


def incident_b0(gamma: float, theta0_deg: float, theta1_deg: float, a1) -> np.ndarray:
    """In-plane incident wavevector: |b0| = gamma cos(theta0), azimuth theta1 from a1."""
    t0 = np.deg2rad(theta0_deg)
    phi = np.arctan2(a1[1], a1[0]) + np.deg2rad(theta1_deg)
    return gamma * np.cos(t0) * np.array([np.cos(phi), np.sin(phi)])


def gamma_squared(gamma: float, b0, k) -> np.ndarray:
    """Gamma_j^2 = gamma^2 - |b0 + k_j|^2 (real)."""
    q = np.asarray(b0)[None, :] + np.asarray(k)
    return gamma * gamma - np.sum(q * q, axis=1)


def gamma_diag(gam2: np.ndarray) -> np.ndarray:
    """Gamma_j with the evanescent branch -i sqrt(|b0+k|^2 - gamma^2) (Im Gamma <= 0)."""
    gam2 = np.asarray(gam2, dtype=np.float64)
    out = np.empty(gam2.shape, dtype=np.complex128)
    pos = gam2 >= 0
    out[pos] = np.sqrt(gam2[pos])
    out[~pos] = -1j * np.sqrt(-gam2[~pos])
    return out


def difference_map(beams):
    """Distinct differences m_j - m_k and the index map l(j, k) into them (Eq. sch2)."""
    b = np.asarray(beams, dtype=np.int64)
    d = b[:, None, :] - b[None, :, :]
    flat = d.reshape(-1, 2)
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    return uniq.astype(np.int64), inv.reshape(b.shape[0], b.shape[0])


class Potential:
    """u_g(z) for the distinct beam differences of a workload, and U(z) = u[l(j,k)](z)."""

    def __init__(self, wl):
        self.wl = wl
        self.diffs, self.lmap = difference_map(wl.beams)
        self.g = rods(self.diffs, wl.a1, wl.a2)                 # (M, 2) cartesian 1/A
        self.g2 = np.sum(self.g * self.g, axis=1)               # (M,)
        a1, a2 = np.asarray(wl.a1, float), np.asarray(wl.a2, float)
        self.area = abs(a1[0] * a2[1] - a1[1] * a2[0])
        self.pref = ((wl.particle - 1j * wl.absorption)
                     * 4.0 * np.pi * lorentz_factor(wl.energy_ev) / self.area)
        self.atoms = np.asarray(wl.atoms, dtype=np.float64)
        sf = np.asarray(wl.sf, dtype=np.float64)[np.asarray(wl.species)]   # (n_atoms, 8)
        self.a = sf[:, :4]                                                  # (n_atoms, 4)
        self.beta = (sf[:, 4:] + np.asarray(wl.dw, dtype=np.float64)[:, None]) / (16.0 * np.pi ** 2)
        # z-independent factor: exp(-i g.r_a) * a_i * exp(-beta |g|^2) / (2 sqrt(pi beta))
        phase = np.exp(-1j * (self.g @ self.atoms[:, :2].T))               # (M, n_atoms)
        amp = self.a[None, :, :] * np.exp(-self.beta[None, :, :] * self.g2[:, None, None]) \
            / (2.0 * np.sqrt(np.pi * self.beta[None, :, :]))                # (M, n_atoms, 4)
        self.F = phase[:, :, None] * amp                                    # (M, n_atoms, 4)
        self._cache = {}

    def u(self, z) -> np.ndarray:
        """u_g(z) for all distinct g: (nz, M) complex; z may be a scalar or array."""
        z = np.atleast_1d(np.asarray(z, dtype=np.float64))
        dz = z[:, None] - self.atoms[None, :, 2]                             # (nz, n_atoms)
        G = np.exp(-dz[:, :, None] ** 2 / (4.0 * self.beta[None, :, :]))   # (nz, n_atoms, 4)
        return self.pref * np.einsum("mak,zak->zm", self.F, G)

    def U(self, z: float) -> np.ndarray:
        key = float(z)
        hit = self._cache.get(key)
        if hit is None:
            hit = self.u(key)[0][self.lmap]
            if len(self._cache) < 200000:
                self._cache[key] = hit
        return hit


class Angle:
    """Per-angle quantities: gamma, b0, Gamma^2 (real) and Gamma (complex, branch Im <= 0)."""

    def __init__(self, wl, theta0_deg: float, theta1_deg: float):
        self.theta0 = float(theta0_deg)
        self.gamma = vacuum_wavenumber(wl.energy_ev)
        self.b0 = incident_b0(self.gamma, theta0_deg, theta1_deg, wl.a1)
        self.k = rods(wl.beams, wl.a1, wl.a2)
        self.gam2 = gamma_squared(self.gamma, self.b0, self.k)
        self.Gam = gamma_diag(self.gam2)


def intensities(rho: np.ndarray, gam2: np.ndarray, theta0_deg: float):
    """eta_i = |rho_i|^2 sin(theta0) Gamma_1 / Gamma_i for propagating beams, else 0.

    Returns (eta, flux) with flux_i = eta_i / sin(theta0) = |rho_i|^2 Gamma_1 / Gamma_i.
    """
    gam2 = np.asarray(gam2, dtype=np.float64)
    prop = gam2 > 0
    flux = np.zeros(gam2.shape)
    g1 = np.sqrt(gam2[0])
    flux[prop] = np.abs(rho[prop]) ** 2 * g1 / np.sqrt(gam2[prop])
    return flux * np.sin(np.deg2rad(theta0_deg)), flux

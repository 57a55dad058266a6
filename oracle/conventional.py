"""Oracle O1: the conventional multi-slice method (Section 2.2 of the paper), plain NumPy FP64.

TEST INFRASTRUCTURE (see ``oracle/model.py``): not used by the CUDA path.

Steps, in the paper's order and notation:

1. Slices z_0 = z_e < z_1 < ... < z_L = 0 of width h; in slice i the coefficient matrix is frozen
   at the midpoint (Eq. ds0): A_i = A((z_i + z_{i+1}) / 2).
2. The slice transfer matrix is the exact exponential A^_i = exp(h A_i) (Eq. ichimiya2). A(z) is
   the tau/rho form of Eq. tr1; it equals S B(z) S^{-1} with B the matrix-ODE coefficient of
   Eq. ode2 and S = [[Gamma, -iI], [Gamma, iI]] (Section 3.1). The exponential is taken through
   the eigendecomposition of M_i = U(m_i) + Gamma^2 (the n x n reduction of the 2n x 2n problem):
   exp(hB) = [[cos(hK), sin(hK)/K], [-K sin(hK), cos(hK)]] as matrix functions of M = K^2.
3. Recursive reflection (Eqs. ri1, ri2): R_{-1} = 0 (rho(z_e) = 0, Eq. bd1),
   R_i = (Z_i + W_i R_{i-1}) (X_i + Y_i R_{i-1})^{-1}, with X, Y, Z, W the n x n blocks of A^_i.
4. rho(0) = R_{L-1} tau(0) with tau(0) = e_1 (Eq. bd0).

Optionally the transmitted wave tau(z_e) = (T_{L-1} ... T_0)^{-1} e_1 with T_i = X_i + Y_i R_{i-1}
(the slice map tau(z_i) -> tau(z_{i+1}) of Eq. ri1's derivation), used by flux-balance tests.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _funcs_of_sqrt(lam: np.ndarray, h: float):
    """cos(h K), sin(h K)/K, K sin(h K) for K = sqrt(lam) (all even in K)."""
    K = np.sqrt(lam.astype(np.complex128))
    small = np.abs(K) < 1e-8
    c = np.cos(h * K)
    s_over_k = np.where(small, h * (1 - (h * K) ** 2 / 6.0), np.sin(h * K) / np.where(small, 1.0, K))
    k_sin = np.where(small, h * lam, K * np.sin(h * K))
    return c, s_over_k, k_sin


def exp_hB(M: np.ndarray, h: float) -> np.ndarray:
    """exp(h B) for B = [[0, I], [-M, 0]] via the eigendecomposition of M (2n x 2n result)."""
    lam, V = np.linalg.eig(M)
    Vinv = np.linalg.inv(V)
    c, sk, ks = _funcs_of_sqrt(lam, h)
    C = (V * c[None, :]) @ Vinv
    Sn = (V * sk[None, :]) @ Vinv
    KS = (V * ks[None, :]) @ Vinv
    n = M.shape[0]
    E = np.empty((2 * n, 2 * n), dtype=np.complex128)
    E[:n, :n] = C
    E[:n, n:] = Sn
    E[n:, :n] = -KS
    E[n:, n:] = C
    return E


def s_matrix(Gam: np.ndarray):
    """S = [[Gamma, -iI], [Gamma, iI]] and its inverse [[(2 Gamma)^-1, (2 Gamma)^-1], [i/2, -i/2]]."""
    n = Gam.shape[0]
    I = np.eye(n)
    S = np.block([[np.diag(Gam), -1j * I], [np.diag(Gam), 1j * I]])
    g2 = np.diag(1.0 / (2.0 * Gam))
    Sinv = np.block([[g2, g2], [0.5j * I, -0.5j * I]])
    return S, Sinv


def a_matrix(Gam: np.ndarray, U: np.ndarray) -> np.ndarray:
    """A(z) of Eq. tr1 written out block by block (used by tests to check S B S^{-1})."""
    n = Gam.shape[0]
    UG = U @ np.diag(1.0 / Gam)
    top = np.hstack([0.5j * UG + 1j * np.diag(Gam), 0.5j * UG])
    bot = np.hstack([-0.5j * UG, -0.5j * UG - 1j * np.diag(Gam)])
    return np.vstack([top, bot])


def slice_transfer(Gam: np.ndarray, gam2: np.ndarray, U: np.ndarray, h: float) -> np.ndarray:
    """A^_i = S exp(h B_i) S^{-1} for the frozen coefficient U (2n x 2n, tau/rho coordinates)."""
    M = U + np.diag(gam2.astype(np.complex128))
    S, Sinv = s_matrix(Gam)
    return S @ exp_hB(M, h) @ Sinv


def rho_conventional(Gam, gam2, Ufun, z_e: float, L: int, transmission: bool = False,
                     expm: bool = False):
    """rho(0) by the conventional multi-slice method with recursive reflection.

    Gam, gam2 : (n,) Gamma and Gamma^2 of one angle; Ufun(z) -> (n, n) complex U(z).
    expm=True takes exp(h A_i) with scipy's Pade scaling-and-squaring instead (cross-check).
    Returns rho (n,) and, with transmission=True, also tau(z_e) (n,).
    """
    n = Gam.shape[0]
    h = -z_e / L
    R = np.zeros((n, n), dtype=np.complex128)
    Ts = []
    for i in range(L):
        z_i = z_e + i * h
        m = z_i + 0.5 * h
        U = Ufun(m)
        if expm:
            Ahat = sla.expm(h * a_matrix(Gam, U + 0.0))
        else:
            Ahat = slice_transfer(Gam, gam2, U, h)
        X, Y = Ahat[:n, :n], Ahat[:n, n:]
        Z, W = Ahat[n:, :n], Ahat[n:, n:]
        T = X + Y @ R
        num = Z + W @ R
        R = np.linalg.solve(T.T, num.T).T
        if transmission:
            Ts.append(T)
    rho = R[:, 0].copy()
    if not transmission:
        return rho
    v = np.zeros(n, dtype=np.complex128)
    v[0] = 1.0
    for T in reversed(Ts):
        v = np.linalg.solve(T, v)
    return rho, v

"""Oracle brute force in high precision (mpmath), for tiny n and L only.

TEST INFRASTRUCTURE (see ``oracle/model.py``): not used by the CUDA path.

* ``rho_direct_product``: the conventional method *without* recursive reflection: the whole-slab
  product A^_{L-1} ... A^_0 of the slice exponentials exp(h A_i) (Eq. ichimiya3), split into
  blocks X^, Y^, Z^, W^, and rho(0) = Z^ X^{-1} tau(0) (Eq. ichimiya4). In FP64 this is the
  ill-conditioned route the paper warns about; at 60+ digits it is a reference for O1.
* ``rho_integrator_no_rhst``: Algorithm 1's ODE loop with the RHST switched off, at 60+ digits,
  then Eq. vrhocomp. It is a reference for O2's RHST (which must not change rho).

The exponentials use mpmath's own ``expm`` on the 2n x 2n tau/rho matrix A(z) of Eq. tr1, an
independent route from O1's eigendecomposition of the n x n matrix M.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

from .integrator import splitting_coefficients


def _mpmat(a):
    a = np.asarray(a)
    M = mp.matrix(a.shape[0], a.shape[1])
    for i in range(a.shape[0]):
        for j in range(a.shape[1]):
            M[i, j] = mp.mpc(complex(a[i, j]))
    return M


def _tonp(M):
    return np.array([[complex(M[i, j]) for j in range(M.cols)] for i in range(M.rows)])


def _a_matrix_mp(Gam, U):
    n = len(Gam)
    A = mp.matrix(2 * n, 2 * n)
    G = [mp.mpc(complex(g)) for g in Gam]
    for j in range(n):
        for k in range(n):
            ug = mp.mpc(complex(U[j, k])) / G[k]
            A[j, k] = 0.5j * ug
            A[j, n + k] = 0.5j * ug
            A[n + j, k] = -0.5j * ug
            A[n + j, n + k] = -0.5j * ug
        A[j, j] += 1j * G[j]
        A[n + j, n + j] -= 1j * G[j]
    return A


def rho_direct_product(Gam, Ufun, z_e: float, L: int, dps: int = 60) -> np.ndarray:
    n = len(Gam)
    with mp.workdps(dps):
        h = mp.mpf(-z_e) / L
        Ptot = mp.eye(2 * n)
        for i in range(L):
            m = z_e + (i + 0.5) * float(-z_e) / L
            A = _a_matrix_mp(Gam, Ufun(m))
            Ptot = mp.expm(h * A) * Ptot
        X = Ptot[0:n, 0:n]
        Z = Ptot[n:2 * n, 0:n]
        e1 = mp.matrix(n, 1)
        e1[0] = 1
        rho = Z * mp.lu_solve(X, e1)
        return np.array([complex(rho[i]) for i in range(n)])


def rho_integrator_no_rhst(Gam, gam2, Ufun, z_e: float, L: int, scheme: str = "sp4",
                           dps: int = 60) -> np.ndarray:
    n = len(Gam)
    a, b = splitting_coefficients(scheme)
    with mp.workdps(dps):
        hf = float(-z_e) / L
        h = mp.mpf(-z_e) / L
        G = [mp.mpc(complex(g)) for g in Gam]
        Q = mp.eye(n)
        P = mp.matrix(n, n)
        for j in range(n):
            P[j, j] = 1j * G[j]
        D = mp.matrix(n, n)
        for j in range(n):
            D[j, j] = mp.mpf(float(gam2[j]))
        for i in range(L):
            z_i = z_e + i * hf
            tau = z_i
            for r in range(len(a)):
                M = _mpmat(Ufun(tau)) + D
                P = P - h * mp.mpf(b[r]) * (M * Q)
                Q = Q + h * mp.mpf(a[r]) * P
                tau = tau + hf * a[r]
            M = _mpmat(Ufun(z_i + hf)) + D
            P = P - h * mp.mpf(b[-1]) * (M * Q)
        GQ = mp.matrix(n, n)
        for j in range(n):
            for k in range(n):
                GQ[j, k] = G[j] * Q[j, k]
        e1 = mp.matrix(n, 1)
        e1[0] = 1
        x = mp.lu_solve(GQ - 1j * P, e1)
        rho = (GQ + 1j * P) * x
        return np.array([complex(rho[i]) for i in range(n)])

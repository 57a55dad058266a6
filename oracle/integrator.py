"""Oracle O2: the proposed method, Algorithm 1 (SolveODE_STR) of the paper, plain NumPy FP64.

TEST INFRASTRUCTURE (see ``oracle/model.py``): not used by the CUDA path.

The state is the economical 2n x n form Z = [Q; P] of Eq. mateq2 (Q = c-block, P = c'-block,
Section 3.1), integrated from z_e to 0 for the matrix ODE Z' = B(z) Z of Eq. ode2 with
B = [[0, I], [-(U + Gamma^2), 0]].

* Initial value: Algorithm 1 starts from S \\ [I; O] = [(2 Gamma)^{-1}; (i/2) I]. By the RHST
  argument of Section 3.2 any right factor leaves rho(0) unchanged, so this oracle starts from
  [I; i Gamma] (the same matrix times 2 Gamma), which needs no Gamma^{-1}.
* One ODE step per slice (Algorithm 1's loop), then the badness xi of Q (after every step, not per
  stage), and the RHST Z <- Z Q^{-1} when xi > threshold (threshold 1000 in Algorithm 1).
* xi is the Gershgorin/Varah bound on the infinity-norm condition number of Q (the paper names
  "Gershgorin" and a guaranteed overestimate but prints no formula):
  xi = max_i sum_j |q_ij| / min_i (|q_ii| - sum_{j != i} |q_ij|), infinite if the
  denominator is not positive.
* rho(0) = (Gamma Q + i P) x with (Gamma Q - i P) x = e_1, which is Eq. vrhocomp multiplied
  through by Q.

Integrators (Section 3.4):

* ``sp4`` / ``sp6``: "BAB" splitting with the SRKN_6^b / SRKN_11^b coefficients of Blanes & Moan
  (2002), which the paper uses but does not print. Section 3.4 names the c-block p and the
  c'-block q (the reverse of Section 3.1's letters); read with p = Q and q = P, stage r = 1..s is
  a kick P <- P - h b_r (U(tau_{r-1}) + Gamma^2) Q, a drift Q <- Q + h a_r P and
  tau_r = tau_{r-1} + h a_r, followed by a last kick with b_{s+1} at tau_s = z_{i+1}.
* ``rk4``: the classical 4-stage Runge-Kutta method applied to Z' = B(z) Z.
* ``magnus2``: the conventional method's step exp(h B(midpoint)) (Section 3.3's bridge between
  the RHST and recursive reflection).
"""
from __future__ import annotations

import numpy as np

from .conventional import exp_hB

# SRKN_6^b: 6 drifts (a1, a2, a3, a3, a2, a1), 7 kicks (b1, b2, b3, b4, b3, b2, b1).
_A6 = (0.209515106613362, -0.143851773179818)
_B6 = (0.0792036964311957, 0.353172906049774, -0.0420650803577195)
# SRKN_11^b: 11 drifts (a1..a5, a6, a5..a1), 12 kicks (b1..b6, b6..b1).
_A11 = (0.123229775946271, 0.290553797799558, -0.127049212625417,
        -0.246331761062075, 0.357208872795928)
_B11 = (0.0414649985182624, 0.198128671918067, -0.0400061921041533,
        0.0752539843015807, -0.0115113874206879)


def splitting_coefficients(scheme: str):
    """(drift coefficients a_1..a_s, kick coefficients b_1..b_{s+1}) of a BAB scheme."""
    if scheme == "sp4":
        a1, a2 = _A6
        a3 = 0.5 - a1 - a2
        b1, b2, b3 = _B6
        b4 = 1.0 - 2.0 * (b1 + b2 + b3)
        return [a1, a2, a3, a3, a2, a1], [b1, b2, b3, b4, b3, b2, b1]
    if scheme == "sp6":
        a = list(_A11)
        a6 = 1.0 - 2.0 * sum(a)
        b = list(_B11)
        b6 = 0.5 - sum(b)
        return a + [a6] + a[::-1], b + [b6, b6] + b[::-1]
    raise ValueError(scheme)


def kick_nodes(scheme: str):
    """Fractions c_r of the step at which the BAB kicks evaluate U (c_0 = 0, ..., c_s = 1)."""
    a, _ = splitting_coefficients(scheme)
    c = [0.0]
    for ar in a:
        c.append(c[-1] + ar)
    return c


def varah(Q: np.ndarray) -> float:
    """Gershgorin/Varah upper bound on the infinity-norm condition number of Q."""
    A = np.abs(Q)
    rows = A.sum(axis=1)
    d = np.diag(A)
    margin = d - (rows - d)
    den = margin.min()
    if not den > 0:
        return np.inf
    return rows.max() / den


def _inside(tau, z_i, h, one_sided):
    # One-sided evaluation for potentials with a jump at a slice boundary: a node on the
    # boundary of step [z_i, z_i + h] takes the value from inside that step.
    if not one_sided:
        return tau
    eps = 1e-12 * h
    return min(max(tau, z_i + eps), z_i + h - eps)


def _bab_step(Q, P, z_i, h, gam2, Ufun, a, b, one_sided=False):
    tau = z_i
    for r in range(len(a)):
        P = P - h * b[r] * ((Ufun(_inside(tau, z_i, h, one_sided)) + np.diag(gam2)) @ Q)
        Q = Q + h * a[r] * P
        tau = tau + h * a[r]
    P = P - h * b[-1] * ((Ufun(_inside(z_i + h, z_i, h, one_sided)) + np.diag(gam2)) @ Q)
    return Q, P


def _rk4_step(Q, P, z_i, h, gam2, Ufun, one_sided=False):
    def f(z, Qs, Ps):
        return Ps, -((Ufun(_inside(z, z_i, h, one_sided)) + np.diag(gam2)) @ Qs)
    k1q, k1p = f(z_i, Q, P)
    k2q, k2p = f(z_i + 0.5 * h, Q + 0.5 * h * k1q, P + 0.5 * h * k1p)
    k3q, k3p = f(z_i + 0.5 * h, Q + 0.5 * h * k2q, P + 0.5 * h * k2p)
    k4q, k4p = f(z_i + h, Q + h * k3q, P + h * k3p)
    Q = Q + (h / 6.0) * (k1q + 2 * k2q + 2 * k3q + k4q)
    P = P + (h / 6.0) * (k1p + 2 * k2p + 2 * k3p + k4p)
    return Q, P


def _magnus2_step(Q, P, z_i, h, gam2, Ufun):
    n = Q.shape[0]
    E = exp_hB(Ufun(z_i + 0.5 * h) + np.diag(gam2.astype(np.complex128)), h)
    Z = E @ np.vstack([Q, P])
    return Z[:n], Z[n:]


def integrate(Gam, gam2, Ufun, z_e: float, L: int, scheme: str = "sp4",
              threshold: float = 1000.0, rhst: bool = True, Z0=None, one_sided: bool = False,
              span=None):
    """Algorithm 1's loop: returns (Q, P, n_rhst) at z = 0 (at z_e + span if ``span`` is given:
    one bulk period for the bulk-layer treatment of Section 2.2).

    Ufun(z) -> (n, n) complex U(z). ``threshold`` is the RHST threshold on xi (xi > threshold
    triggers Z <- Z Q^{-1}); ``rhst=False`` disables the transform altogether. ``one_sided``
    evaluates U at a step's end points from inside the step (for potentials with jumps exactly
    at slice boundaries; smooth potentials do not need it).
    """
    n = Gam.shape[0]
    h = (-z_e if span is None else float(span)) / L
    gam2 = np.asarray(gam2, dtype=np.float64)
    if Z0 is None:
        Q = np.eye(n, dtype=np.complex128)
        P = np.diag(1j * Gam)
    else:
        Q, P = Z0[:n].astype(np.complex128), Z0[n:].astype(np.complex128)
    if scheme in ("sp4", "sp6"):
        a, b = splitting_coefficients(scheme)
    n_rhst = 0
    for i in range(L):
        z_i = z_e + i * h
        if scheme in ("sp4", "sp6"):
            Q, P = _bab_step(Q, P, z_i, h, gam2, Ufun, a, b, one_sided)
        elif scheme == "rk4":
            Q, P = _rk4_step(Q, P, z_i, h, gam2, Ufun, one_sided)
        elif scheme == "magnus2":
            Q, P = _magnus2_step(Q, P, z_i, h, gam2, Ufun)
        else:
            raise ValueError(scheme)
        if rhst and varah(Q) > threshold:
            P = np.linalg.solve(Q.T, P.T).T
            Q = np.eye(n, dtype=np.complex128)
            n_rhst += 1
    return Q, P, n_rhst


def assemble(Gam, Q, P) -> np.ndarray:
    """rho(0) = (Gamma Q + i P) x, (Gamma Q - i P) x = e_1 (Eq. vrhocomp times Q)."""
    n = Gam.shape[0]
    GQ = Gam[:, None] * Q
    e1 = np.zeros(n, dtype=np.complex128)
    e1[0] = 1.0
    x = np.linalg.solve(GQ - 1j * P, e1)
    return (GQ + 1j * P) @ x


def rho_integrator(Gam, gam2, Ufun, z_e: float, L: int, scheme: str = "sp4",
                   threshold: float = 1000.0, rhst: bool = True, one_sided: bool = False):
    """rho(0) by Algorithm 1; returns (rho, n_rhst)."""
    Q, P, n_rhst = integrate(Gam, gam2, Ufun, z_e, L, scheme, threshold, rhst,
                             one_sided=one_sided)
    return assemble(Gam, Q, P), n_rhst

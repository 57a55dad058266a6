"""Closed forms used to pin the oracle (one beam, uniform slab).

TEST INFRASTRUCTURE (see ``oracle/model.py``).

One beam (n = 1, k_1 = 0), a uniform potential U0 on -d < z < 0 and vacuum elsewhere. With
K = sqrt(Gamma^2 + U0) and the paper's tau/rho decomposition (Eqs. vtau, vrho: the incident wave
is exp(i Gamma z), tau(0) = 1, rho(z_e) = 0), matching c and c' at z = 0 and z = -d gives

    rho(0) = -i U0 sin(K d) / (2 Gamma K cos(K d) + i (Gamma^2 + K^2) sin(K d)),

which is even in K. For a thick absorbing slab (Im K < 0) it tends to (Gamma - K)/(Gamma + K).
"""
from __future__ import annotations

import numpy as np


def slab_rho(Gam: complex, U0: complex, d: float) -> complex:
    K = np.sqrt(complex(Gam) ** 2 + complex(U0))
    s, c = np.sin(K * d), np.cos(K * d)
    return -1j * U0 * s / (2.0 * Gam * K * c + 1j * (Gam ** 2 + K ** 2) * s)


def half_space_rho(Gam: complex, U0: complex) -> complex:
    K = np.sqrt(complex(Gam) ** 2 + complex(U0))
    if K.imag > 0:
        K = -K
    return (Gam - K) / (Gam + K)

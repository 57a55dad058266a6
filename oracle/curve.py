"""Oracle rocking curves: the forward model over a batch of glancing angles (Section 2.1).

TEST INFRASTRUCTURE (see ``oracle/model.py``): not used by the CUDA path.

``rocking_curve`` runs O2 (Algorithm 1) or O1 (the conventional method) for every angle of a
workload and returns rho (A, n), eta (A, n), flux (A, n) and the RHST counts. U(z) is built once
per structure and shared by all angles (Section 3.4: the same U(z) serves every angle).
``rocking_curve_parallel`` spreads angles over a ``spawn`` process pool with one BLAS thread per
process.
"""
from __future__ import annotations

import os

import numpy as np

from .conventional import rho_conventional
from .integrator import rho_integrator
from .model import Angle, Potential, intensities


def angle_solve(wl, pot: Potential, theta0: float, theta1: float, method: str = "sp4",
                threshold: float = 1000.0, n_steps=None):
    ang = Angle(wl, theta0, theta1)
    L = wl.n_steps if n_steps is None else int(n_steps)
    if method == "conventional":
        rho = rho_conventional(ang.Gam, ang.gam2, pot.U, wl.z_e, L)
        n_rhst = 0
    else:
        rho, n_rhst = rho_integrator(ang.Gam, ang.gam2, pot.U, wl.z_e, L, method, threshold)
    eta, flux = intensities(rho, ang.gam2, theta0)
    return rho, eta, flux, n_rhst


def rocking_curve(wl, method: str = "sp4", threshold: float = 1000.0, angles=None,
                  n_steps=None, pot: Potential = None):
    pot = Potential(wl) if pot is None else pot
    idx = range(len(wl.theta0)) if angles is None else angles
    rhos, etas, fluxes, counts = [], [], [], []
    for a in idx:
        rho, eta, flux, n = angle_solve(wl, pot, wl.theta0[a], wl.theta1[a], method, threshold,
                                        n_steps)
        rhos.append(rho)
        etas.append(eta)
        fluxes.append(flux)
        counts.append(n)
    return np.array(rhos), np.array(etas), np.array(fluxes), np.array(counts)


def _worker(args):
    wl, a, method, threshold, n_steps = args
    pot = Potential(wl)
    return rocking_curve(wl, method, threshold, [a], n_steps, pot)


_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def rocking_curve_parallel(wl, method: str = "sp4", threshold: float = 1000.0, angles=None,
                           n_steps=None, processes=None):
    """Angles spread over a spawn-started process pool (one angle per task)."""
    import multiprocessing as mpc
    idx = list(range(len(wl.theta0))) if angles is None else list(angles)
    procs = processes or len(os.sched_getaffinity(0))
    ctx = mpc.get_context("spawn")
    # children read the BLAS thread count when they import NumPy, i.e. from the environment
    # they inherit at spawn time
    saved = {v: os.environ.get(v) for v in _BLAS_VARS}
    for v in _BLAS_VARS:
        os.environ[v] = "1"
    try:
        with ctx.Pool(min(procs, len(idx))) as pool:
            parts = pool.map(_worker, [(wl, a, method, threshold, n_steps) for a in idx],
                             chunksize=1)
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(4))


def curve_error(eta, eta_ref) -> float:
    """eacc-style error of a rocking curve (Section 4): max over angles of the Euclidean norm of
    the intensity difference over beams, divided by the max over angles of the reference norm."""
    eta, eta_ref = np.atleast_2d(eta), np.atleast_2d(eta_ref)
    num = np.max(np.linalg.norm(eta - eta_ref, axis=1))
    den = np.max(np.linalg.norm(eta_ref, axis=1))
    return float(num / den)

"""Oracle for the reverse analysis: the R-factor of a rocking curve and its gradient with respect
to atomic z coordinates and Debye-Waller classes, by central finite differences of O2.

TEST INFRASTRUCTURE (see ``oracle/model.py``): not used by the CUDA path.

The paper fits structures by minimising the disagreement between measured and computed rocking
curves (Section 1, reverse analysis) but prints no R-factor formula, so this oracle takes the
plain reading: the rocking curve is the specular intensity eta_1(theta) over the glancing angles,
normalised to unit sum, and

    R = sum_theta (eta~(theta) - eta~_target(theta))^2,   eta~ = eta_1 / sum_theta eta_1.

Its gradient here is the plain definition of a derivative, evaluated by central differences of
Algorithm 1 (O2) in FP64:

    dR/dp ~ (R(p + h) - R(p - h)) / (2 h),

for each parameter p: the z coordinate of each free atom (h in Angstrom) and the B factor shared
by all atoms of a Debye-Waller class (h in Angstrom^2). The same evaluations give the Jacobian of
the specular curve, d eta_1(theta) / dp. Curves are computed over a spawn-started process pool
(one BLAS thread per process), one task per (perturbed structure, angle).
"""
from __future__ import annotations

import os
from dataclasses import replace

import numpy as np

from .curve import _BLAS_VARS
from .integrator import rho_integrator
from .model import Angle, Potential, intensities


def normalized(curve) -> np.ndarray:
    c = np.asarray(curve, dtype=np.float64)
    return c / c.sum(axis=-1, keepdims=True)


def rfactor(eta1, target) -> float:
    """R = sum over angles of the squared difference of the unit-sum normalised curves."""
    return float(np.sum((normalized(eta1) - normalized(target)) ** 2))


def perturbed(wl, free_atoms, dw_class, k: int, delta: float):
    """The structure with parameter k moved by delta: k < n_free moves z of free_atoms[k];
    k >= n_free adds delta to B of every atom in Debye-Waller class k - n_free."""
    n_free = len(free_atoms)
    if k < n_free:
        atoms = np.array(wl.atoms, dtype=np.float64, copy=True)
        atoms[free_atoms[k], 2] += delta
        return replace(wl, atoms=atoms)
    dw = np.array(wl.dw, dtype=np.float64, copy=True)
    dw[np.asarray(dw_class) == (k - n_free)] += delta
    return replace(wl, dw=dw)


def _eta1_task(args):
    wl, a, threshold = args
    pot = Potential(wl)
    ang = Angle(wl, wl.theta0[a], wl.theta1[a])
    rho, _ = rho_integrator(ang.Gam, ang.gam2, pot.U, wl.z_e, wl.n_steps, "sp4", threshold)
    eta, _ = intensities(rho, ang.gam2, wl.theta0[a])
    return eta[0]


def specular_curves(structures, threshold: float = 1000.0, processes=None) -> np.ndarray:
    """eta_1(theta) of each structure over its angles: (n_structures, n_angles)."""
    import multiprocessing as mpc
    tasks = [(wl, a, threshold) for wl in structures for a in range(len(wl.theta0))]
    procs = min(processes or len(os.sched_getaffinity(0)), len(tasks))
    if procs <= 1:
        out = [_eta1_task(t) for t in tasks]
    else:
        saved = {v: os.environ.get(v) for v in _BLAS_VARS}
        for v in _BLAS_VARS:
            os.environ[v] = "1"
        try:
            with mpc.get_context("spawn").Pool(procs) as pool:
                out = pool.map(_eta1_task, tasks, chunksize=1)
        finally:
            for v, val in saved.items():
                if val is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = val
    return np.asarray(out, dtype=np.float64).reshape(len(structures), -1)


def fd_gradient(wl, free_atoms, dw_class, target, hz: float = 1e-5, hb: float = 1e-5,
                threshold: float = 1000.0, processes=None):
    """Central differences of O2 at the structure ``wl``.

    Returns a dict with R, eta1 (n_angles,), grad (n_free + n_classes,) = dR/dp and
    jac (n_angles, n_free + n_classes) = d eta_1 / dp. ``dw_class`` holds a class index per atom
    (-1: B fixed); the classes are 0 .. max(dw_class).
    """
    free_atoms = np.asarray(free_atoms, dtype=np.int64)
    dw_class = np.asarray(dw_class, dtype=np.int64)
    n_free = len(free_atoms)
    n_par = n_free + int(dw_class.max()) + 1 if dw_class.size and dw_class.max() >= 0 else n_free
    steps = [hz if k < n_free else hb for k in range(n_par)]
    structures = [wl]
    for k in range(n_par):
        structures.append(perturbed(wl, free_atoms, dw_class, k, +steps[k]))
        structures.append(perturbed(wl, free_atoms, dw_class, k, -steps[k]))
    curves = specular_curves(structures, threshold, processes)
    eta1 = curves[0]
    grad = np.empty(n_par)
    jac = np.empty((len(eta1), n_par))
    for k in range(n_par):
        cp, cm = curves[1 + 2 * k], curves[2 + 2 * k]
        grad[k] = (rfactor(cp, target) - rfactor(cm, target)) / (2.0 * steps[k])
        jac[:, k] = (cp - cm) / (2.0 * steps[k])
    return {"R": rfactor(eta1, target), "eta1": eta1, "grad": grad, "jac": jac}

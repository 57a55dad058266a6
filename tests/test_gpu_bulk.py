"""Bulk layer on the GPU (Section 2.2, end): the converged bulk boundary condition, computed once
per set of directions and reused, against the oracle (oracle/bulk.py)."""
import numpy as np
import pytest

from oracle import bulk as B
from oracle.curve import curve_error
from paper_2306_00271_gb300 import workloads as W

pytestmark = pytest.mark.gpu
PERIOD, STEPS = 2.4, 48


@pytest.fixture(scope="module")
def api():
    from paper_2306_00271_gb300 import api as a
    a.load()
    return a


def _case(n_beams=7, seed=5):
    wl = W.tiny(n_beams=n_beams, seed=seed, n_steps=60, theta0=(0.8, 1.9, 3.4), depth=6.0,
                absorption=0.6)
    atoms = np.array([[0.7, 0.4, -1.1], [2.1, 1.5, -2.0]])
    return wl, atoms, np.array([0.5, 0.7]), np.zeros(2, dtype=np.int32)


def _oracle(wl, atoms, dw, sp):
    out = [B.angle_bulk(wl, atoms, dw, sp, PERIOD, STEPS, t0, t1)
           for t0, t1 in zip(wl.theta0, wl.theta1)]
    return (np.array([o[2] for o in out]), np.array([o[3] for o in out]),
            max(o[1] for o in out))


@pytest.mark.parametrize("n_beams", [7, 19])
def test_bulk_fp64_against_oracle(api, n_beams):
    wl, atoms, dw, sp = _case(n_beams)
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_bulk(atoms, dw, sp, PERIOD, STEPS)
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    st = eng.stats()
    rho_o, eta_o, k_o = _oracle(wl, atoms, dw, sp)
    assert curve_error(eta.cpu().numpy()[0], eta_o) <= 1e-10
    assert np.max(np.abs(rho.cpu().numpy()[0] - rho_o)) <= 1e-10 * np.max(np.abs(rho_o))
    assert abs(st["bulk_periods"] - k_o) <= 1 and st["ms_bulk"] > 0
    # the bulk changes the curve (it is not the no-wave start)
    _, eta_free = api.Engine(wl, "fp64", "sp4").rocking_curve(wl.theta0, wl.theta1)
    assert curve_error(eta_free.cpu().numpy()[0], eta_o) > 1e-6
    # same directions again: the cached boundary condition is reused
    eng.rocking_curve(wl.theta0, wl.theta1)
    assert eng.stats()["bulk_periods"] == 0


@pytest.mark.parametrize("n_beams", [19, 37])
def test_bulk_mixed_against_oracle(api, n_beams):
    wl, atoms, dw, sp = _case(n_beams)
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_column_split("on")  # two CTAs per pair when N > 32: the split form starts from [I; X]
    eng.set_bulk(atoms, dw, sp, PERIOD, STEPS)
    _, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    assert eng.stats()["column_split"] == (1 if n_beams > 32 else 0)
    _, eta_o, _ = _oracle(wl, atoms, dw, sp)
    assert curve_error(eta.cpu().numpy()[0], eta_o) <= 1e-6


def test_bulk_gradient_matches_differences(api):
    """The bulk is fixed, so the slab's gradient starts from the constant [I; X_bulk]; check the
    reverse sweep against central differences of the GPU forward (FP64, h = 1e-5)."""
    wl, atoms, dw, sp = _case(7)
    free, cls = np.array([0, 1, 2, 3]), np.array([0, 0, 1, 1])
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_bulk(atoms, dw, sp, PERIOD, STEPS)
    eng.set_fit(free, cls, ckpt_every=16)
    _, jac = eng.curve_jacobian(wl.theta0, wl.theta1)
    jac = jac.cpu().numpy()[0]
    fd = np.empty_like(jac)
    h = 1e-5
    for k in range(len(free) + 2):
        curves = []
        for sgn in (1, -1):
            at, d = wl.atoms.copy(), wl.dw.copy()
            if k < len(free):
                at[free[k], 2] += sgn * h
            else:
                d[cls == k - len(free)] += sgn * h
            eng.set_structures(at[None], d[None])
            curves.append(eng.rocking_curve(wl.theta0, wl.theta1)[1].cpu().numpy()[0][:, 0])
        fd[:, k] = (curves[0] - curves[1]) / (2 * h)
    assert np.max(np.abs(jac - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_bulk_in_a_batch_and_no_convergence(api):
    wl, atoms, dw, sp = _case(7)
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_bulk(atoms, dw, sp, PERIOD, STEPS)
    _, eta_s = eng.rocking_curve(wl.theta0, wl.theta1)
    eng2 = api.Engine(wl, "fp64", "sp4")
    eng2.set_bulk(atoms, dw, sp, PERIOD, STEPS)
    batch = api.Batch()
    _, eta_b = batch.add(eng2, wl.theta0, wl.theta1)
    batch.run()
    e_s, e_b = eta_s.cpu().numpy(), eta_b.cpu().numpy()
    assert np.max(np.abs(e_b - e_s)) <= 1e-11 * np.max(np.abs(e_s))
    batch.close()
    bad = api.Engine(wl, "fp64", "sp4")
    bad.set_bulk(atoms, dw, sp, PERIOD, STEPS, max_periods=3, tol=1e-15)
    with pytest.raises(api.TrhError) as e:
        bad.rocking_curve(wl.theta0, wl.theta1)
    assert e.value.code == api.TRH_ENOCONV

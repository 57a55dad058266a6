"""Pins for the R-factor oracle and its finite-difference gradient (oracle/gradient.py)."""
import numpy as np
import pytest

from oracle import gradient as G
from paper_2306_00271_gb300 import workloads as W


def test_rfactor_hand_example():
    # curve (1,2,3,4)/10 against a flat target 1/4: differences -0.15, -0.05, 0.05, 0.15
    assert G.rfactor([1.0, 2.0, 3.0, 4.0], [2.0, 2.0, 2.0, 2.0]) == pytest.approx(0.05, rel=1e-15)


def test_rfactor_zero_at_target_and_scale_free():
    rng = np.random.default_rng(5)
    c, t = rng.uniform(0.1, 1.0, 60), rng.uniform(0.1, 1.0, 60)
    assert G.rfactor(c, c) == 0.0
    assert G.rfactor(3.7 * c, 0.2 * t) == pytest.approx(G.rfactor(c, t), rel=1e-14)
    assert G.rfactor(c, t) > 0.0


def test_perturbed_moves_exactly_one_parameter():
    wl = W.tiny(n_beams=3, n_steps=10)
    cls = np.array([0, 0, 1, -1])
    z = G.perturbed(wl, [1, 3], cls, 1, 0.25)
    assert np.array_equal(z.atoms[:, 2] - wl.atoms[:, 2], [0, 0, 0, 0.25])
    assert np.array_equal(z.dw, wl.dw)
    b = G.perturbed(wl, [1, 3], cls, 2, 0.1)      # class 0 = atoms 0 and 1
    assert np.allclose(b.dw - wl.dw, [0.1, 0.1, 0, 0], rtol=0, atol=1e-15)
    assert np.array_equal(b.atoms, wl.atoms)


def _eta1_brute(wl):
    from oracle.brute import rho_integrator_no_rhst
    from oracle.model import Angle, Potential
    pot = Potential(wl)
    ang = Angle(wl, wl.theta0[0], wl.theta1[0])
    rho = rho_integrator_no_rhst(ang.Gam, ang.gam2, pot.U, wl.z_e, wl.n_steps, "sp4", dps=40)
    return abs(rho[0]) ** 2 * np.sin(np.deg2rad(wl.theta0[0]))


def test_fd_jacobian_matches_high_precision_five_point_derivative():
    """Brute force on a tiny input: O2 without the RHST at 40 digits, differentiated with a
    five-point stencil at a step 100x larger (truncation O(h^4)), against the FP64 central
    differences of O2 with the RHST."""
    wl = W.tiny(n_beams=3, n_steps=16, seed=11, depth=5.0, theta0=(2.2,))
    free = np.array([0, 2, 3])
    cls = np.array([0, 1, 1, 0])
    fd = G.fd_gradient(wl, free, cls, target=np.ones(1), processes=1)
    hs = 1e-3
    ref = []
    for k in range(len(free) + 2):
        f = [_eta1_brute(G.perturbed(wl, free, cls, k, m * hs)) for m in (2, 1, -1, -2)]
        ref.append((-f[0] + 8 * f[1] - 8 * f[2] + f[3]) / (12 * hs))
    ref = np.array(ref)
    assert np.max(np.abs(fd["jac"][0] - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert np.all(np.abs(ref) > 1e-4 * np.max(np.abs(ref)))   # every parameter matters here


def test_class_derivative_is_sum_of_member_derivatives():
    wl = W.tiny(n_beams=3, n_steps=12, seed=3, depth=5.0, theta0=(1.8,))
    free = np.array([], dtype=np.int64)
    pair = G.fd_gradient(wl, free, np.array([0, 0, -1, -1]), np.ones(1), processes=1)["jac"][0]
    single = G.fd_gradient(wl, free, np.array([0, 1, -1, -1]), np.ones(1), processes=1)["jac"][0]
    assert pair[0] == pytest.approx(single[0] + single[1], rel=1e-7)


def test_fd_gradient_converges_with_step():
    """Central differences are O(h^2): the gradients at h and h/2 agree far below the 1e-5
    tolerance the CUDA adjoint is held to."""
    wl = W.tiny(n_beams=4, n_steps=20, seed=4, depth=6.0, theta0=(1.0, 2.0, 3.0))
    free, cls = np.array([0, 1]), np.array([0, 0, 1, 1])
    target = np.array([0.3, 0.2, 0.1])
    g1 = G.fd_gradient(wl, free, cls, target, hz=1e-4, hb=1e-4, processes=1)["grad"]
    g2 = G.fd_gradient(wl, free, cls, target, hz=5e-5, hb=5e-5, processes=1)["grad"]
    assert np.max(np.abs(g1 - g2)) <= 1e-6 * np.max(np.abs(g2))


def test_rfactor_gradient_is_chain_rule_of_jacobian():
    """dR/dp from differences of R equals the chain rule through the normalised curve applied
    to the Jacobian from differences of eta_1."""
    wl = W.tiny(n_beams=3, n_steps=12, seed=9, depth=5.0, theta0=(1.2, 2.4))
    free, cls = np.array([1, 2]), np.array([-1, 0, 0, -1])
    target = np.array([0.02, 0.05])
    fd = G.fd_gradient(wl, free, cls, target, processes=1)
    e, t = fd["eta1"], target / target.sum()
    S = e.sum()
    r = e / S - t
    dR_deta = 2 * r / S - 2 * np.dot(r, e) / S ** 2
    assert np.allclose(fd["grad"], dR_deta @ fd["jac"], rtol=1e-6, atol=1e-9 * np.abs(fd["grad"]).max())

"""Reverse sweep (adjoint of Algorithm 1 on the FP64 path) vs the oracle's central differences.

Bar: gradients within 1e-5 relative (max abs difference over parameters / max abs oracle
gradient); the oracle's central differences themselves agree with a 40-digit five-point
derivative to ~1e-10 (tests/test_oracle_gradient.py), so the bar is set by the CUDA path."""
import os

import numpy as np
import pytest

from oracle import gradient as G
from paper_2306_00271_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rfactor_fit_n61.npz")
TOL = 1e-5


@pytest.fixture(scope="module")
def api():
    from paper_2306_00271_gb300 import api as a
    a.load()
    return a


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _small():
    # 37 beams (three 16-row tiles and a ragged tail), 240 steps over a 12 A slab: dozens of
    # RHSTs, and with checkpoints every 32 steps eight segments of which the last is ragged
    return W.tiny(n_beams=37, n_steps=240, seed=31, depth=12.0, theta0=(0.6, 1.4, 2.9, 4.1))


def test_jacobian_matches_oracle_differences(api):
    wl = _small()
    free, cls = np.array([0, 1, 2, 3]), np.array([0, 1, 1, 0])
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(free, cls, ckpt_every=32)
    eta, jac = eng.curve_jacobian(wl.theta0, wl.theta1)
    fd = G.fd_gradient(wl, free, cls, target=np.ones(len(wl.theta0)))
    jac = jac.cpu().numpy()[0]
    assert jac.shape == fd["jac"].shape
    assert _rel(jac, fd["jac"]) <= 1e-6, _rel(jac, fd["jac"])
    assert np.allclose(eta.cpu().numpy()[0][:, 0], fd["eta1"], rtol=1e-10, atol=0)
    st = eng.stats()
    assert st["rhst_total"] > 10 * len(wl.theta0) and st["ms_gradient"] > 0
    assert st["column_split"] == 1   # 4 angles: the forward ran with two CTAs per angle
    assert st["sweep_split"] == 1    # and so did the reverse sweep's recompute and adjoint
    # the one-CTA forward and sweep: the same trajectory and the same adjoint bit for bit, so the
    # same curve and the same Jacobian (to the order of the contraction's atomic additions)
    eng.set_column_split("off")
    eta1, jac1 = eng.curve_jacobian(wl.theta0, wl.theta1)
    assert eng.stats()["column_split"] == 0 and eng.stats()["sweep_split"] == 0
    assert np.array_equal(eta1.cpu().numpy(), eta.cpu().numpy())
    assert _rel(jac1.cpu().numpy()[0], jac) <= 1e-12


def test_checkpoint_interval_does_not_change_the_gradient(api):
    wl = _small()
    free, cls = np.array([0, 2]), np.array([-1, 0, 0, -1])
    eng = api.Engine(wl, "fp64", "sp4")
    out = []
    for C in (7, 64, 240, 1000):
        eng.set_fit(free, cls, ckpt_every=C)
        out.append(eng.curve_jacobian(wl.theta0, wl.theta1)[1].cpu().numpy())
    for o in out[1:]:
        assert _rel(o, out[0]) <= 1e-12


def test_rfactor_gradient_small(api):
    wl = _small()
    free, cls = np.array([1, 3]), np.array([0, 0, 1, 1])
    target = np.array([0.05, 0.02, 0.01, 0.004])
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(free, cls, ckpt_every=50)
    R, gz, gb = eng.rfactor_grad(wl.theta0, wl.theta1, target)
    fd = G.fd_gradient(wl, free, cls, target)
    g = np.concatenate([gz.cpu().numpy()[0], gb.cpu().numpy()[0]])
    assert float(R[0]) == pytest.approx(fd["R"], rel=1e-10)
    assert _rel(g, fd["grad"]) <= 1e-6, _rel(g, fd["grad"])


def test_parameter_sets_are_independent(api):
    wl = W.tiny(n_beams=13, n_steps=120, seed=5, depth=9.0, theta0=(1.0, 2.0, 3.0))
    free, cls = np.array([0, 1, 2]), np.array([0, 0, 1, 1])
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(free, cls, ckpt_every=40)
    a2 = wl.atoms.copy()
    a2[:, 2] -= 0.3
    dw2 = wl.dw + 0.2
    eng.set_structures(np.stack([wl.atoms, a2]), np.stack([wl.dw, dw2]))
    _, jac2 = eng.curve_jacobian(wl.theta0, wl.theta1)
    for k, (at, dw) in enumerate(((wl.atoms, wl.dw), (a2, dw2))):
        eng.set_structures(at[None], dw[None])
        _, jac1 = eng.curve_jacobian(wl.theta0, wl.theta1)
        assert _rel(jac2.cpu().numpy()[k], jac1.cpu().numpy()[0]) <= 1e-13


def test_full_size_rfactor_gradient_matches_golden(api):
    """12 surface z and 6 Debye-Waller classes at N = 61, 2000 slices, 60 angles, checkpoints
    every 64 steps; target and gradient from the oracle (tests/golden/make_golden_grad.py)."""
    gold = np.load(GOLDEN)
    fp = W.rfactor_fit()
    wl = fp.workload
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(fp.free_atoms, fp.dw_class, ckpt_every=64)
    R, gz, gb = eng.rfactor_grad(wl.theta0, wl.theta1, gold["target"])
    g = np.concatenate([gz.cpu().numpy()[0], gb.cpu().numpy()[0]])
    assert float(R[0]) == pytest.approx(float(gold["R"]), rel=1e-9)
    assert _rel(g, gold["grad"]) <= TOL, _rel(g, gold["grad"])
    st = eng.stats()
    assert st["n_bad"] == 0 and st["kernels_launched"] >= 3 * 32


def test_autograd_function(api):
    import torch
    wl = W.tiny(n_beams=13, n_steps=100, seed=8, depth=8.0, theta0=(0.9, 1.7, 2.6))
    free, cls = np.array([0, 3]), np.array([0, -1, 0, 1])
    target = np.array([0.03, 0.01, 0.02])
    eng = api.Engine(wl, "fp64", "sp4")
    fit = api.RFactor(eng, free, cls, wl.theta0, wl.theta1, target, ckpt_every=25)
    z = torch.tensor(wl.atoms[free, 2][None], dtype=torch.float64, device="cuda",
                     requires_grad=True)
    b = torch.tensor([[wl.dw[0], wl.dw[3]]], dtype=torch.float64, device="cuda",
                     requires_grad=True)
    R = fit(z, b)
    (2.0 * R.sum()).backward()
    fd = G.fd_gradient(wl, free, cls, target)
    assert float(R[0]) == pytest.approx(fd["R"], rel=1e-10)
    g = np.concatenate([z.grad.cpu().numpy()[0], b.grad.cpu().numpy()[0]])
    assert _rel(g, 2.0 * fd["grad"]) <= 1e-6


def test_fit_argument_errors(api):
    wl = W.tiny(n_beams=3, n_steps=10)
    eng = api.Engine(wl, "fp64", "sp4")
    t0, t1, jac = np.array([1.5]), np.array([0.0]), np.zeros(8)
    code = eng.lib.trh_curve_jacobian(eng.ctx, 1, api._ptr(t0), api._ptr(t1), None,
                                      api._ptr(jac), None)
    assert code == api.TRH_EINVAL            # no trh_set_fit yet
    for free, cls in (([7], None), ([0, 0], None), ([], [0, 2, -1, -1]), ([], None)):
        with pytest.raises(api.TrhError) as e:
            eng.set_fit(free, cls)
        assert e.value.code == api.TRH_EINVAL


def test_mixed_forward_gradient(api):
    """A mixed-precision context: forward and checkpoints on the mixed path, segments recomputed
    in binary64; small size against the oracle's central differences and full size against the
    golden gradient, both within the 1e-5 bar."""
    wl = _small()
    free, cls = np.array([1, 3]), np.array([0, 0, 1, 1])
    target = np.array([0.05, 0.02, 0.01, 0.004])
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_fit(free, cls, ckpt_every=50)
    R, gz, gb = eng.rfactor_grad(wl.theta0, wl.theta1, target)
    fd = G.fd_gradient(wl, free, cls, target)
    g = np.concatenate([gz.cpu().numpy()[0], gb.cpu().numpy()[0]])
    assert float(R[0]) == pytest.approx(fd["R"], rel=1e-6)
    assert _rel(g, fd["grad"]) <= TOL, _rel(g, fd["grad"])
    gold = np.load(GOLDEN)
    fp = W.rfactor_fit()
    eng = api.Engine(fp.workload, "mixed", "sp4")
    eng.set_fit(fp.free_atoms, fp.dw_class, ckpt_every=64)
    R, gz, gb = eng.rfactor_grad(fp.workload.theta0, fp.workload.theta1, gold["target"])
    g = np.concatenate([gz.cpu().numpy()[0], gb.cpu().numpy()[0]])
    assert _rel(g, gold["grad"]) <= TOL, _rel(g, gold["grad"])
    st = eng.stats()
    assert st["ms_integrate"] < 1000.0      # the forward ran on the mixed path


def test_mixed_jacobian_digit_contraction(api):
    """A mixed context of <= 64 beams forms each kick's Ubar on the tensor cores from four-digit
    operands (the recompute and the adjoint stay binary64): its Jacobian agrees with the oracle's
    central differences within the bar and with a binary64 context's Jacobian to ~1e-7, the
    FP32-level rounding of the digit products summed over kicks. Ragged N (37: a 74 x 74 product
    in a 128 x 128 tile) and a ragged last segment; the checkpoint interval changes nothing but
    the order of the contraction's atomic additions."""
    wl = _small()
    free, cls = np.array([0, 1, 2, 3]), np.array([0, 1, 1, 0])
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_fit(free, cls, ckpt_every=32)
    eta, jac = eng.curve_jacobian(wl.theta0, wl.theta1)
    jac = jac.cpu().numpy()[0]
    fd = G.fd_gradient(wl, free, cls, target=np.ones(len(wl.theta0)))
    assert _rel(jac, fd["jac"]) <= TOL, _rel(jac, fd["jac"])
    ref = api.Engine(wl, "fp64", "sp4")
    ref.set_fit(free, cls, ckpt_every=32)
    jac64 = ref.curve_jacobian(wl.theta0, wl.theta1)[1].cpu().numpy()[0]
    assert 0.0 < _rel(jac, jac64) <= 1e-6, _rel(jac, jac64)
    eng.set_fit(free, cls, ckpt_every=7)
    jac7 = eng.curve_jacobian(wl.theta0, wl.theta1)[1].cpu().numpy()[0]
    assert _rel(jac7, jac) <= 1e-6


@pytest.mark.parametrize("n_beams, n_steps, depth", [(11, 60, 4.0), (64, 40, 3.0)])
def test_mixed_jacobian_edge_sizes(api, n_beams, n_steps, depth):
    """The digit contraction at its shape limits: 11 beams (a 22 x 22 product, two K-steps, one
    CTA per angle in the sweep) and 64 beams (2N = 128 fills the tile's rows, the leading digit's
    MMA is 256 columns wide): the mixed context's Jacobian against the binary64 context's."""
    wl = W.tiny(n_beams=n_beams, n_steps=n_steps, seed=41, depth=depth, theta0=(0.9, 2.4))
    free, cls = np.array([0, 2]), np.array([0, 0, 1, 1])
    out = {}
    for prec in ("mixed", "fp64"):
        eng = api.Engine(wl, prec, "sp4")
        eng.set_fit(free, cls, ckpt_every=16)
        out[prec] = eng.curve_jacobian(wl.theta0, wl.theta1)[1].cpu().numpy()[0]
        assert eng.stats()["sweep_split"] == (1 if n_beams > 32 else 0)
    assert np.all(np.isfinite(out["mixed"])) and np.max(np.abs(out["fp64"])) > 0
    assert _rel(out["mixed"], out["fp64"]) <= 1e-6, _rel(out["mixed"], out["fp64"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_wide_jacobian_matches_oracle_differences(api, precision):
    """70 beams (64 < N <= 256): the wide reverse sweep (state in global memory, products on the
    FP64 tensor pipe in tiles, the contraction folded into the adjoint kernel) against the
    oracle's central differences, with a ragged last segment. On a mixed context the forward of a
    gradient above 64 beams also runs in binary64, so both precisions give this Jacobian."""
    wl = W.tiny(n_beams=70, n_steps=60, seed=33, depth=6.0, theta0=(0.8, 2.2, 3.5))
    free, cls = np.array([0, 1, 2, 3]), np.array([0, 1, 1, 0])
    eng = api.Engine(wl, precision, "sp4")
    eng.set_fit(free, cls, ckpt_every=16)
    eta, jac = eng.curve_jacobian(wl.theta0, wl.theta1)
    fd = G.fd_gradient(wl, free, cls, target=np.ones(len(wl.theta0)))
    jac = jac.cpu().numpy()[0]
    assert _rel(jac, fd["jac"]) <= 1e-6, _rel(jac, fd["jac"])
    assert np.allclose(eta.cpu().numpy()[0][:, 0], fd["eta1"], rtol=1e-10, atol=0)
    st = eng.stats()
    assert st["rhst_total"] > 0 and st["ms_gradient"] > 0 and st["wide_tile"] in (32, 64)
    eng.set_fit(free, cls, ckpt_every=7)
    jac7 = eng.curve_jacobian(wl.theta0, wl.theta1)[1].cpu().numpy()[0]
    assert _rel(jac7, jac) <= 1e-12


def test_wide_rfactor_gradient(api):
    """The R-factor and its gradient through trh_rfactor_grad at 91 beams against the oracle's
    central differences of R."""
    wl = W.tiny(n_beams=91, n_steps=40, seed=35, depth=5.0, theta0=(0.9, 1.8, 2.6, 3.9))
    free, cls = np.array([1, 3]), np.array([0, 0, 1, 1])
    target = np.array([0.2, 0.3, 0.25, 0.25])
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(free, cls, ckpt_every=16)
    R, gz, gb = eng.rfactor_grad(wl.theta0, wl.theta1, target)
    fd = G.fd_gradient(wl, free, cls, target=target)
    got = np.concatenate([np.asarray(gz.cpu()).ravel(), np.asarray(gb.cpu()).ravel()])
    want = fd["grad"]
    assert float(np.asarray(R.cpu()).ravel()[0]) == pytest.approx(fd["R"], rel=1e-10)
    assert _rel(got, want) <= 1e-5, _rel(got, want)


def test_wide_jacobian_150_beams(api):
    """150 beams (three 64-column blocks with a ragged last one): the wide reverse sweep's
    Jacobian against the oracle's central differences on a thin slab."""
    wl = W.tiny(n_beams=150, n_steps=16, seed=37, depth=2.5, theta0=(1.1, 2.4))
    free, cls = np.array([0]), np.array([0, 0, -1, -1])
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(free, cls, ckpt_every=6)
    _, jac = eng.curve_jacobian(wl.theta0, wl.theta1)
    fd = G.fd_gradient(wl, free, cls, target=np.ones(len(wl.theta0)))
    assert _rel(jac.cpu().numpy()[0], fd["jac"]) <= 1e-6

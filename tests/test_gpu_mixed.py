"""Mixed-precision CUDA path (tensor-core kicks on four-digit fixed-point BF16 operands,
double-float state, FP32 RHST inverse applied in double-float, FP64 assembly with one refinement
step) vs the oracle's Algorithm 1, with one and with two CTAs per angle.

Bar: <= 1e-6 per rocking curve (eacc-style, as in the FP64 tests); rho elementwise within 1e-6
of the curve's largest |rho|."""
import os

import numpy as np
import pytest

from oracle.curve import curve_error, rocking_curve
from paper_2306_00271_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "trhepd_n61_sp4.npz")
TOL = 1e-6


@pytest.fixture(scope="module")
def api():
    from paper_2306_00271_gb300 import api as a
    a.load()
    return a


def _check(rho_g, eta_g, rho_o, eta_o, tol=TOL):
    rho_g = np.asarray(rho_g).reshape(rho_o.shape)
    eta_g = np.asarray(eta_g).reshape(eta_o.shape)
    assert np.all(np.isfinite(rho_g))
    err = curve_error(eta_g, eta_o)
    assert err <= tol, err
    assert np.max(np.abs(rho_g - rho_o)) <= tol * np.max(np.abs(rho_o))
    return err


def test_rheed_row_single_angle(api):
    wl = W.rheed_row()
    eng = api.Engine(wl, "mixed", "sp4")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho_o, eta_o, _, n_o = rocking_curve(wl, "sp4")
    _check(rho.cpu().numpy()[0], eta.cpu().numpy()[0], rho_o, eta_o)
    st = eng.stats()
    assert st["n_bad"] == 0 and st["rhst_total"] > 0


@pytest.mark.parametrize("n_beams", [1, 2, 3, 7, 13, 19, 37, 64])
def test_ragged_beam_counts(api, n_beams):
    wl = W.tiny(n_beams=n_beams, seed=20 + n_beams, n_steps=60, theta0=(0.7, 1.9, 3.3),
                depth=8.0)
    eng = api.Engine(wl, "mixed", "sp4")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho_o, eta_o, _, _ = rocking_curve(wl, "sp4")
    _check(rho.cpu().numpy()[0], eta.cpu().numpy()[0], rho_o, eta_o)


def test_sp6_scheme(api):
    wl = W.tiny(n_beams=19, seed=4, n_steps=40, theta0=(1.1, 2.7), depth=8.0)
    eng = api.Engine(wl, "mixed", "sp6")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho_o, eta_o, _, _ = rocking_curve(wl, "sp6")
    _check(rho.cpu().numpy()[0], eta.cpu().numpy()[0], rho_o, eta_o)


def test_several_parameter_sets(api):
    sets = W.batch_sets(3, beam_classes=(61,))
    wl = sets[0].with_steps(150).with_angles([0.9, 2.4, 5.1])
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_structures(np.stack([s.atoms for s in sets]))
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    for k, s in enumerate(sets):
        wk = s.with_steps(150).with_angles([0.9, 2.4, 5.1])
        rho_o, eta_o, _, _ = rocking_curve(wk, "sp4")
        _check(rho.cpu().numpy()[k], eta.cpu().numpy()[k], rho_o, eta_o)


def test_mixed_matches_fp64_path(api):
    wl = W.tiny(n_beams=37, seed=9, n_steps=300, theta0=(0.8, 2.2, 4.4), depth=10.0)
    r_m, e_m = api.Engine(wl, "mixed", "sp4").rocking_curve(wl.theta0, wl.theta1)
    r_d, e_d = api.Engine(wl, "fp64", "sp4").rocking_curve(wl.theta0, wl.theta1)
    assert curve_error(e_m.cpu().numpy()[0], e_d.cpu().numpy()[0]) <= TOL


@pytest.mark.parametrize("n_beams", [33, 48, 61, 64])
def test_column_split_matches_one_cta(api, n_beams):
    """Two CTAs per pair (a cluster sharing the columns) against one CTA per pair: the same
    arithmetic per column and the same order of the Varah row sums, so the same RHST steps and
    the same curve to rounding; both against the oracle."""
    wl = W.tiny(n_beams=n_beams, seed=40 + n_beams, n_steps=160,
                theta0=(0.6, 1.4, 2.9, 4.4), depth=10.0)
    out = {}
    for mode in ("on", "off"):
        eng = api.Engine(wl, "mixed", "sp4")
        eng.set_column_split(mode)
        rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
        st = eng.stats()
        assert st["column_split"] == (1 if mode == "on" else 0) and st["n_bad"] == 0
        out[mode] = (rho.cpu().numpy()[0], eta.cpu().numpy()[0], st["rhst_total"])
    assert out["on"][2] == out["off"][2] > 0
    assert np.max(np.abs(out["on"][0] - out["off"][0])) <= 1e-12 * np.max(np.abs(out["off"][0]))
    rho_o, eta_o, _, _ = rocking_curve(wl, "sp4")
    _check(out["on"][0], out["on"][1], rho_o, eta_o)


def test_column_split_modes(api):
    wl = W.tiny(n_beams=19, seed=3, n_steps=20, theta0=(1.0,), depth=4.0)
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_column_split("on")   # 19 beams: one CTA owns every column, no split
    eng.rocking_curve(wl.theta0, wl.theta1)
    assert eng.stats()["column_split"] == 0
    assert eng.lib.trh_set_column_split(eng.ctx, 7) == api.TRH_EINVAL


@pytest.mark.parametrize("mode", ["auto", "off"])
def test_full_rocking_curve_61_beams(api, mode):
    """Full size (61 beams, 2000 slices, 60 angles), the launch the benchmark times (auto: two
    CTAs per angle on a device with at least 120 SMs), and the one-CTA form."""
    wl = W.trhepd_n61()
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_column_split(mode)
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    if mode == "off":
        assert eng.stats()["column_split"] == 0
    rho, eta = rho.cpu().numpy()[0], eta.cpu().numpy()[0]
    if os.path.exists(GOLDEN):
        g = np.load(GOLDEN)
        _check(rho, eta, g["rho"], g["eta"])
    else:
        idx = [0, 15, 37, 59]
        rho_o, eta_o, _, _ = rocking_curve(wl, "sp4", angles=idx)
        _check(rho[idx], eta[idx], rho_o, eta_o)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotuned_split_matches_both_forms(api, precision):
    """TRH_SPLIT_AUTO: the autotuner times both forms on a probe of the call's pairs and keeps the
    faster (trh_stats.tuned = 1); the curve equals the forced one-CTA and two-CTA curves bitwise,
    and a second call with the same shape reuses the cached choice."""
    wl = W.tiny(n_beams=45, seed=17, n_steps=30, theta0=(0.7, 1.6, 2.9, 4.1), depth=6.0)
    out = {}
    for mode in ("off", "on", "auto"):
        eng = api.Engine(wl, precision, "sp4")
        eng.set_column_split(mode)
        rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
        st = eng.stats()
        out[mode] = (rho.cpu().numpy(), st)
        if mode == "auto":
            assert st["tuned"] == 1
            rho2, _ = eng.rocking_curve(wl.theta0, wl.theta1)
            assert eng.stats()["tuned"] == 1
            assert eng.stats()["column_split"] == st["column_split"]
            assert np.array_equal(rho2.cpu().numpy(), out[mode][0])
        else:
            assert st["tuned"] == 0
        eng.close()
    assert out["off"][1]["column_split"] == 0 and out["on"][1]["column_split"] == 1
    assert np.array_equal(out["off"][0], out["on"][0])
    assert np.array_equal(out["auto"][0], out["off"][0])


def test_autotuner_picks_the_split_for_a_long_curve(api):
    """60 angles of 61 beams at 400 slices: the two-CTA form is about 1.7x faster per step there,
    and the tuner, extrapolating its 2- and 12-step probes to the call's 400 steps, picks it."""
    wl = W.trhepd_n61().with_steps(400)
    eng = api.Engine(wl, "mixed", "sp4")
    eng.rocking_curve(wl.theta0, wl.theta1)
    st = eng.stats()
    assert st["tuned"] == 1 and st["column_split"] == 1

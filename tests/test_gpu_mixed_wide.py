"""Mixed-precision CUDA path for wide beam sets (64 < N <= 128): a thread-block cluster of
ceil(N / 32) CTAs per (set, angle) pair, tensor-core digit products streamed per node, double-float
state, FP32 RHST inverse applied in double-float, binary64 assembly. Against the oracle's
Algorithm 1 and against the FP64 wide kernel, through the C ABI.

Bar: <= 1e-6 per rocking curve (eacc-style) and rho elementwise within 1e-6 of the curve's largest
|rho|, as for the N <= 64 mixed path."""
import numpy as np
import pytest

from oracle.curve import curve_error, rocking_curve, rocking_curve_parallel
from oracle import model
from paper_2306_00271_gb300 import workloads as W

pytestmark = pytest.mark.gpu
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


@pytest.mark.parametrize("n_beams", [65, 91, 97, 121, 128])
def test_ragged_beam_counts_against_oracle(api, n_beams):
    """Cluster sizes 3 and 4, ragged last CTA (65, 97: one live column in it), K padded with
    zero slices (ceil(2N / 16) = 9 -> 12, 13 -> 16) and the largest N."""
    wl = W.tiny(n_beams=n_beams, seed=80 + n_beams, n_steps=40, theta0=(0.8, 2.6), depth=8.0)
    eng = api.Engine(wl, "mixed", "sp4")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho_o, eta_o, _, n_o = rocking_curve(wl, "sp4")
    _check(rho.cpu().numpy()[0], eta.cpu().numpy()[0], rho_o, eta_o)
    st = eng.stats()
    assert st["ctas_per_pair"] == (n_beams + 31) // 32
    assert st["n_bad"] == 0 and st["rhst_total"] > 0
    # the FP32 Varah bound may cross the threshold a step earlier or later than the binary64 one
    assert abs(st["rhst_total"] - int(n_o.sum())) <= 4


def test_sp6_scheme(api):
    wl = W.tiny(n_beams=77, seed=5, n_steps=30, theta0=(1.3,), depth=6.0)
    eng = api.Engine(wl, "mixed", "sp6")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho_o, eta_o, _, _ = rocking_curve(wl, "sp6")
    _check(rho.cpu().numpy()[0], eta.cpu().numpy()[0], rho_o, eta_o)


def test_121_beam_sets_against_oracle(api):
    """The 121-beam class of the batched workload: two perturbed structures in one call."""
    sets = [s for s in W.batch_sets(6) if s.beams.shape[0] == 121]
    wl = sets[0].with_steps(60).with_angles([1.2, 3.4])
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_structures(np.stack([s.atoms for s in sets]))
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    for k, s in enumerate(sets):
        rho_o, eta_o, _, _ = rocking_curve(s.with_steps(60).with_angles([1.2, 3.4]), "sp4")
        _check(rho.cpu().numpy()[k], eta.cpu().numpy()[k], rho_o, eta_o)


def test_121_beams_full_depth_sampled_angles(api):
    """A 121-beam structure of the batched workload at its full 2000 slices of 0.015 A, in the
    launch configuration of a whole curve (60 angles, one cluster each), checked against the
    oracle on two sampled angles and against the FP64 wide kernel on all of them."""
    wl = [s for s in W.batch_sets(3) if s.beams.shape[0] == 121][0]
    assert wl.n_steps == 2000 and len(wl.theta0) == 60
    eng = api.Engine(wl, "mixed", "sp4")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho, eta = rho.cpu().numpy()[0], eta.cpu().numpy()[0]
    idx = [7, 41]
    rho_o, eta_o, _, _ = rocking_curve_parallel(wl, "sp4", angles=idx, processes=2)
    _check(rho[idx], eta[idx], rho_o, eta_o)
    ref = api.Engine(wl, "fp64", "sp4")
    rho_f, eta_f = ref.rocking_curve(wl.theta0, wl.theta1)
    _check(rho, eta, rho_f.cpu().numpy()[0], eta_f.cpu().numpy()[0])


def test_set_chunks_give_the_same_curves(api):
    """Three structures whose images exceed a small budget run in three chunks of one set; the
    arithmetic per pair is the same, so the curves are bitwise those of one chunk. (0.3 A steps:
    at 1.5 A the fastest evanescent beams of this beam set grow by ~e^16 within one step, beyond
    what the FP32 RHST inverse handles, and the mixed path reports TRH_ESINGULAR.)"""
    sets = [s for s in W.batch_sets(9) if s.beams.shape[0] == 121]
    wl = sets[0].with_steps(100).with_angles([1.0, 2.2, 5.0])
    atoms = np.stack([s.atoms for s in sets])
    out = {}
    for budget in (0, 1):
        eng = api.Engine(wl, "mixed", "sp4")
        eng.set_image_budget(budget)
        eng.set_structures(atoms)
        rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
        out[budget] = (rho.cpu().numpy(), eng.stats()["set_chunks"])
    assert out[0][1] == 1 and out[1][1] == 3
    assert np.array_equal(out[0][0], out[1][0])


def test_narrow_mixed_set_chunks(api):
    """The same for the N <= 64 mixed kernel (two CTAs per pair and one)."""
    wl = W.tiny(n_beams=37, seed=9, n_steps=30, theta0=(0.9, 2.9), depth=6.0)
    rng = np.random.default_rng(5)
    atoms = np.stack([wl.atoms.copy() for _ in range(3)])
    atoms[..., 2] = np.minimum(atoms[..., 2] + rng.normal(0, 0.05, atoms.shape[:2]), 0.0)
    out = {}
    for budget in (0, 1):
        eng = api.Engine(wl, "mixed", "sp4")
        eng.set_image_budget(budget)
        eng.set_structures(atoms)
        rho, _ = eng.rocking_curve(wl.theta0, wl.theta1)
        out[budget] = (rho.cpu().numpy(), eng.stats()["set_chunks"])
    assert out[0][1] == 1 and out[1][1] == 3
    assert np.array_equal(out[0][0], out[1][0])


def test_in_a_batch_with_other_beam_counts(api):
    """A 97-beam mixed job beside 37-beam mixed and 19-beam FP64 jobs in one batch (eager run,
    then graph replay) equals the standalone curves."""
    wls = [W.tiny(n_beams=n, seed=90 + n, n_steps=30, theta0=(1.1, 2.8), depth=6.0)
           for n in (97, 37, 19)]
    precs = ["mixed", "mixed", "fp64"]
    engines = [api.Engine(w, p, "sp4") for w, p in zip(wls, precs)]
    batch = api.Batch()
    outs = [batch.add(e, w.theta0, w.theta1) for e, w in zip(engines, wls)]
    for run in range(2):
        batch.run()
        st = batch.stats()
        assert st["graph_replay"] == run and st["n_bad"] == 0
        for (rho_b, _), e, w in zip(outs, engines, wls):
            rho_s, _ = e.rocking_curve(w.theta0, w.theta1)
            np.testing.assert_array_equal(rho_b.cpu().numpy(), rho_s.cpu().numpy())
    batch.close()


def test_grazing_beam_ends_only_its_pair(api):
    """A beam exactly on the Ewald circle: every CTA of that pair's cluster sees it and the pair
    reports TRH_EGRAZING with NaN outputs; the other angle of the call is unaffected."""
    import torch
    wl = W.tiny(n_beams=70, seed=2, n_steps=20, depth=4.0, theta0=(1.0,))
    gamma = model.vacuum_wavenumber(wl.energy_ev)
    k = model.rods(wl.beams, wl.a1, wl.a2)
    j = int(np.argmax(k[:, 0]))
    theta = float(np.rad2deg(np.arccos((-k[j, 0] + np.sqrt(gamma ** 2 - k[j, 1] ** 2)) / gamma)))
    assert abs(model.Angle(wl, theta, 0.0).gam2[j]) < 1e-9
    eng = api.Engine(wl, "mixed", "sp4")
    eta = torch.empty((1, 2, 70), dtype=torch.float64, device="cuda")
    with pytest.raises(api.TrhError) as ei:
        eng.rocking_curve([theta, 2.0], [0.0, 0.0], eta=eta)
    assert ei.value.code == api.TRH_EGRAZING
    st = eng.stats()
    assert st["n_bad"] == 1 and st["first_bad_angle"] == 0
    e = eta.cpu().numpy()[0]
    assert np.all(np.isnan(e[0])) and np.all(np.isfinite(e[1]))


def test_limits(api):
    wl = W.tiny(n_beams=257, seed=1, n_steps=4)
    with pytest.raises(api.TrhError) as e:
        api.Engine(wl, "mixed", "sp4")
    assert e.value.code == api.TRH_EUNSUPPORTED


def test_chunked_batch_equals_standalone(api):
    """Mixed jobs of 121 beams (3 structures) and 37 beams (2 structures) beside an FP64 job,
    with an image budget that forces one chunk per structure: the batch builds each chunk's
    images and integrates it inside its launch sequence; the eager run and the graph replay
    equal the standalone curves bitwise."""
    sets = [s for s in W.batch_sets(9) if s.beams.shape[0] == 121]
    w121 = sets[0].with_steps(100).with_angles([1.0, 3.0])
    w37 = W.tiny(n_beams=37, seed=11, n_steps=40, theta0=(0.9, 2.7), depth=6.0)
    w19 = W.tiny(n_beams=19, seed=12, n_steps=40, theta0=(1.3,), depth=6.0)
    e121 = api.Engine(w121, "mixed", "sp4")
    e121.set_structures(np.stack([s.atoms for s in sets]))
    e37 = api.Engine(w37, "mixed", "sp4")
    a37 = np.stack([w37.atoms, w37.atoms + np.array([0.0, 0.0, -0.05])])
    e37.set_structures(a37)
    e19 = api.Engine(w19, "fp64", "sp4")
    for e in (e121, e37):
        e.set_image_budget(1)
    batch = api.Batch()
    outs = [batch.add(e, w.theta0, w.theta1) for e, w in ((e121, w121), (e37, w37), (e19, w19))]
    for run in range(2):
        batch.run()
        st = batch.stats()
        assert st["graph_replay"] == run and st["n_bad"] == 0
        assert st["set_chunks"] == 3
        for (rho_b, _), (e, w) in zip(outs, ((e121, w121), (e37, w37), (e19, w19))):
            rho_s, _ = e.rocking_curve(w.theta0, w.theta1)
            np.testing.assert_array_equal(rho_b.cpu().numpy(), rho_s.cpu().numpy())
    batch.close()

"""Mixed-precision CUDA path for the widest beam sets (128 < N <= 256): a thread-block cluster of
ceil(N / 16) CTAs per (set, angle) pair, tensor-core digit tiles built in shared memory from a
per-node digit table on the grid of beam differences, double-float state, FP32 RHST inverse by a
Gauss-Jordan elimination distributed over the cluster and applied in double-float, binary64
assembly. Against the oracle's Algorithm 1 and against the FP64 wide kernel, through the C ABI.

Bar: <= 1e-6 per rocking curve (eacc-style) and rho elementwise within 1e-6 of the curve's largest
|rho|, as for the narrower mixed paths."""
from dataclasses import replace

import numpy as np
import pytest

from oracle.curve import curve_error, rocking_curve
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


@pytest.mark.parametrize("n_beams", [129, 150, 192, 200, 255])
def test_ragged_beam_counts_against_oracle(api, n_beams):
    """Cluster sizes 9 to 16 (129: one live column in the last CTA), three and four row tiles
    (2N = 384 fills three exactly), K padded to an even count of 16-wide slices."""
    wl = W.tiny(n_beams=n_beams, seed=90 + n_beams, n_steps=40, theta0=(0.9, 2.7), depth=8.0)
    eng = api.Engine(wl, "mixed", "sp4")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho_o, eta_o, _, n_o = rocking_curve(wl, "sp4")
    _check(rho.cpu().numpy()[0], eta.cpu().numpy()[0], rho_o, eta_o)
    st = eng.stats()
    assert st["ctas_per_pair"] == (n_beams + 15) // 16
    assert st["n_bad"] == 0 and st["rhst_total"] > 0
    # the FP32 Varah bound may cross the threshold a step earlier or later than the binary64 one
    assert abs(st["rhst_total"] - int(n_o.sum())) <= 4


def test_sp6_and_two_structures(api):
    """The SRKN_11^b scheme, and two parameter sets in one call (one launch, grid y = sets)."""
    wl = W.tiny(n_beams=170, seed=11, n_steps=24, theta0=(1.4, 3.1), depth=6.0)
    atoms2 = wl.atoms.copy()
    atoms2[:, 2] -= 0.2
    eng = api.Engine(wl, "mixed", "sp6")
    eng.set_structures(np.stack([wl.atoms, atoms2]))
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    for k, at in enumerate([wl.atoms, atoms2]):
        w2 = replace(wl, atoms=at)
        rho_o, eta_o, _, _ = rocking_curve(w2, "sp6")
        _check(rho.cpu().numpy()[k], eta.cpu().numpy()[k], rho_o, eta_o)


def test_against_fp64_wide_kernel(api):
    """The 255-beam square cell of the large recipe on a 6 A slab: every angle of a 16-angle
    sweep against the FP64 wide kernel."""
    wl = W.large_n255(1)[0]
    wl = replace(wl, z_e=-6.0).with_steps(120).with_angles(
        np.linspace(0.3, 6.0, 16))
    mixed = api.Engine(wl, "mixed", "sp4")
    fp64 = api.Engine(wl, "fp64", "sp4")
    rho_m, eta_m = mixed.rocking_curve(wl.theta0, wl.theta1)
    rho_f, eta_f = fp64.rocking_curve(wl.theta0, wl.theta1)
    _check(rho_m.cpu().numpy()[0], eta_m.cpu().numpy()[0], rho_f.cpu().numpy()[0],
           eta_f.cpu().numpy()[0])
    assert mixed.stats()["ctas_per_pair"] == 16


def test_set_chunks_are_bitwise_equal(api):
    """Sets split into chunks (an image budget of one set's digit tables) give the same bits as
    one chunk."""
    wl = W.tiny(n_beams=140, seed=3, n_steps=20, theta0=(1.0, 2.2), depth=5.0)
    atoms = np.stack([wl.atoms, wl.atoms + np.array([0.0, 0.0, -0.1])])
    one = api.Engine(wl, "mixed", "sp4")
    one.set_structures(atoms)
    rho1, eta1 = one.rocking_curve(wl.theta0, wl.theta1)
    two = api.Engine(wl, "mixed", "sp4")
    two.set_structures(atoms)
    two.set_image_budget(1)
    rho2, eta2 = two.rocking_curve(wl.theta0, wl.theta1)
    assert two.stats()["set_chunks"] == 2
    assert np.array_equal(rho1.cpu().numpy(), rho2.cpu().numpy())
    assert np.array_equal(eta1.cpu().numpy(), eta2.cpu().numpy())


def test_grazing_beam_ends_only_its_pair(api):
    """A beam exactly on the Ewald circle: every CTA of that pair's cluster sees it and the pair
    reports TRH_EGRAZING with NaN outputs; the other angle of the call is unaffected."""
    import torch
    from oracle import model
    wl = W.tiny(n_beams=140, seed=4, n_steps=16, depth=5.0, theta0=(1.0,))
    gamma = model.vacuum_wavenumber(wl.energy_ev)
    k = model.rods(wl.beams, wl.a1, wl.a2)
    j = int(np.argmax(k[:, 0]))
    theta = float(np.rad2deg(np.arccos((-k[j, 0] + np.sqrt(gamma ** 2 - k[j, 1] ** 2)) / gamma)))
    assert abs(model.Angle(wl, theta, 0.0).gam2[j]) < 1e-9
    eng = api.Engine(wl, "mixed", "sp4")
    eta = torch.empty((1, 2, 140), dtype=torch.float64, device="cuda")
    with pytest.raises(api.TrhError) as ei:
        eng.rocking_curve([theta, 2.0], [0.0, 0.0], eta=eta)
    assert ei.value.code == api.TRH_EGRAZING
    st = eng.stats()
    assert st["n_bad"] == 1 and st["first_bad_angle"] == 0
    e = eta.cpu().numpy()[0]
    assert np.all(np.isnan(e[0])) and np.all(np.isfinite(e[1]))


def test_limits(api):
    """A beam set whose difference grid exceeds the shared-memory table is refused at creation."""
    a1, a2 = W.square_lattice(5.4)
    beams = np.array([[0, 0], [1, 0], [0, 1]] + [[m, 40] for m in range(-70, 70)], dtype=np.int32)
    wl = replace(W.tiny(n_beams=3, seed=1, n_steps=4), beams=beams, a1=a1, a2=a2)
    with pytest.raises(api.TrhError) as e:
        api.Engine(wl, "mixed", "sp4")
    assert e.value.code == api.TRH_EUNSUPPORTED


def test_large_recipe_full_depth_sampled_angles(api):
    """The 255-beam recipe's first structure at its full 3000 slices of 0.01 A, all 120 angles in
    one call (the launch configuration of the bench line), against the oracle's curve at the
    sampled angles stored in tests/golden (written by make_golden.py from the oracle alone)."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "large_n255_sp4_sampled.npz"))
    wl = W.large_n255(1)[0]
    assert wl.n_steps == int(g["n_steps"]) and len(wl.theta0) == 120
    np.testing.assert_array_equal(wl.theta0[g["angles"]], g["theta0"])
    eng = api.Engine(wl, "mixed", "sp4")
    rho, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    rho, eta = rho.cpu().numpy()[0], eta.cpu().numpy()[0]
    assert np.all(np.isfinite(rho)) and eng.stats()["n_bad"] == 0
    _check(rho[g["angles"]], eta[g["angles"]], g["rho"], g["eta"])


def test_batch_with_a_wide_job_equals_standalone(api):
    """A batch holding a 140-beam mixed job (16-column CTAs in a cluster of 9) beside a 37-beam
    mixed job and an FP64 job: the eager run and the graph replay equal the standalone curves
    bitwise."""
    w140 = W.tiny(n_beams=140, seed=21, n_steps=20, theta0=(1.2, 2.8), depth=5.0)
    w37 = W.tiny(n_beams=37, seed=22, n_steps=30, theta0=(0.9, 2.1, 3.3), depth=6.0)
    w19 = W.tiny(n_beams=19, seed=23, n_steps=30, theta0=(1.5,), depth=6.0)
    e140 = api.Engine(w140, "mixed", "sp4")
    e140.set_structures(np.stack([w140.atoms, w140.atoms + np.array([0.0, 0.0, -0.1])]))
    e37 = api.Engine(w37, "mixed", "sp4")
    e19 = api.Engine(w19, "fp64", "sp4")
    batch = api.Batch()
    jobs = ((e140, w140), (e37, w37), (e19, w19))
    outs = [batch.add(e, w.theta0, w.theta1) for e, w in jobs]
    for run in range(2):
        batch.run()
        st = batch.stats()
        assert st["graph_replay"] == run and st["n_bad"] == 0
        for (rho_b, eta_b), (e, w) in zip(outs, jobs):
            rho_s, eta_s = e.rocking_curve(w.theta0, w.theta1)
            np.testing.assert_array_equal(rho_b.cpu().numpy(), rho_s.cpu().numpy())
            np.testing.assert_array_equal(eta_b.cpu().numpy(), eta_s.cpu().numpy())
    batch.close()

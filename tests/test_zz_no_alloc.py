"""The no-allocation entry point, for callers that cannot call cudaMalloc when they need a curve:
code under a fixed device-memory budget that must not grow, plug-ins whose host application owns
all device memory, and loops where cudaMalloc's implicit synchronisation is not acceptable. It
must give the same binary64 rocking curve as the context-based entry point, on two calls in a row
that share the library's fixed device array, for both splitting schemes and beam counts on both
sides of 32 (one or two CTAs' worth of columns), and must refuse problems whose tables do not fit
that array. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2306_00271_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10  # the binary64 path's tolerance


def _run_twice(wl, integrator, angle_lists):
    import torch

    from oracle.curve import curve_error
    from paper_2306_00271_gb300 import api
    api.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    eng = api.Engine(wl, "fp64", integrator)
    for theta0 in angle_lists:
        t0 = torch.tensor(theta0, dtype=torch.float64, device=dev)
        t1 = torch.full_like(t0, float(wl.theta1[0]))
        rho = torch.empty((len(theta0), wl.n_beams), dtype=torch.complex128, device=dev)
        eta = torch.empty((len(theta0), wl.n_beams), dtype=torch.float64, device=dev)
        api.rocking_curve_noalloc(wl, t0, t1, rho, eta, integrator=integrator)
        torch.cuda.synchronize()
        ref_rho, ref_eta = eng.rocking_curve(t0, t1)
        ref_rho, ref_eta = ref_rho.cpu().numpy()[0], ref_eta.cpu().numpy()[0]
        got_rho, got_eta = rho.cpu().numpy(), eta.cpu().numpy()
        assert np.all(np.isfinite(got_rho))
        assert np.max(np.abs(got_rho - ref_rho)) <= TOL * np.max(np.abs(ref_rho))
        assert curve_error(got_eta, ref_eta) <= TOL
    eng.close()


@pytest.mark.parametrize("integrator", ["sp4", "sp6"])
def test_noalloc_matches_context_entry_on_two_calls(integrator):
    wl = W.rheed_row()  # 11 beams, 400 slices: tables well inside the fixed array
    _run_twice(wl, integrator, ([2.0], [1.2, 2.5, 3.7]))


@pytest.mark.parametrize("integrator", ["sp4", "sp6"])
def test_noalloc_61_beams(integrator):
    """61 beams (217 distinct differences) at 100 slices: 601 (sp4) or 1101 (sp6) nodes x 217 x
    16 B, inside the 16 MiB array."""
    wl = W.trhepd_n61().with_steps(100)
    _run_twice(wl, integrator, ([0.9, 3.3], [1.7]))


def test_noalloc_rejects_tables_beyond_its_array():
    import torch

    from paper_2306_00271_gb300 import api
    api.load()
    wl = W.trhepd_n61()  # 12001 nodes x 217 differences x 16 B = 41.7 MB > 16 MiB
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = torch.tensor([2.0], dtype=torch.float64, device=dev)
    rho = torch.empty((1, wl.n_beams), dtype=torch.complex128, device=dev)
    eta = torch.empty((1, wl.n_beams), dtype=torch.float64, device=dev)
    with pytest.raises(api.TrhError) as ei:
        api.rocking_curve_noalloc(wl, t0, torch.zeros_like(t0), rho, eta)
    assert ei.value.code == api.TRH_EINVAL
    assert "bytes of scratch" in str(ei.value)

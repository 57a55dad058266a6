"""Step-size sweep: accuracy against time for the integrators (Section 4's time-error study).

For each method (the conventional multi-slice method of Section 2.2 as the comparison point, and
Algorithm 1 with sp4 = SRKN_6^b, sp6 = SRKN_11^b, rk4) and precision path, the slab is
integrated at the step sizes dz of the E-6 series 0.010 ... 0.68 A, and the rocking curve's error
is measured against a fine reference (sp6, FP64, half the smallest step) with the paper's
curve error: the maximum over angles of the Euclidean norm of the intensity difference over
beams, divided by the maximum over angles of the reference norm. Time is the integration kernel's
device time per curve (CUDA events, no table build).

    python -m paper_2306_00271_gb300.sweep [--workload trhepd_n61] [--angles 60] [--out FILE]
        [--column-split auto|on|off]

The splitting integrators can run two CTAs per angle (column split, `Engine.set_column_split`);
the conventional method runs one. The table records which.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import workloads as W

E6 = (0.010, 0.015, 0.022, 0.033, 0.047, 0.068, 0.10, 0.15, 0.22, 0.33, 0.47, 0.68)


def curve_error(eta, ref) -> float:
    eta, ref = np.atleast_2d(eta), np.atleast_2d(ref)
    return float(np.max(np.linalg.norm(eta - ref, axis=1)) / np.max(np.linalg.norm(ref, axis=1)))


def _curve(api, wl, precision, integrator, split="auto"):
    """(eta, device ms of the integration kernel, RHST count, failed pairs). A step too coarse
    for the fastest evanescent beams can overflow Q within one step; the library reports that
    as a singular pivot and returns NaN for those angles."""
    import torch
    eng = api.Engine(wl, precision, integrator)
    eng.set_column_split(split)
    eta = torch.empty((1, len(wl.theta0), eng.N), dtype=torch.float64, device="cuda")
    try:
        eng.rocking_curve(wl.theta0, wl.theta1, eta=eta)
    except api.TrhError:
        pass   # the failed angles are NaN; the count is in the stats
    st = eng.stats()
    eng.close()
    return eta.cpu().numpy()[0], st["ms_integrate"], st["rhst_total"], st["n_bad"], \
        1 + st["column_split"]


def run(workload: str = "trhepd_n61", n_angles: int = 60, runs=None, split: str = "auto"):
    import torch
    from . import api
    api.load()
    base = W.RECIPES[workload]()
    idx = np.linspace(0, len(base.theta0) - 1, min(n_angles, len(base.theta0))).round().astype(int)
    base = base.with_angles(base.theta0[idx], base.theta1[idx])
    depth = -base.z_e
    ref_L = int(round(depth / (E6[0] / 2)))
    ref, ref_ms, _, _, _ = _curve(api, base.with_steps(ref_L), "fp64", "sp6", split)
    runs = runs or [("fp64", "conventional"), ("fp64", "sp4"), ("fp64", "sp6"), ("fp64", "rk4"),
                    ("mixed", "sp4"), ("mixed", "sp6")]
    rows = []
    for precision, integrator in runs:
        for dz in E6:
            L = max(1, int(round(depth / dz)))
            t = time.perf_counter()
            eta, ms, nr, bad, ctas = _curve(api, base.with_steps(L), precision, integrator, split)
            ok = np.all(np.isfinite(eta))
            rows.append(dict(precision=precision, integrator=integrator, dz=depth / L, L=L,
                             err=curve_error(eta, ref) if ok else float("nan"), ms=ms, rhst=nr,
                             failed=bad, ctas=ctas, wall=time.perf_counter() - t))
            torch.cuda.synchronize()
    return dict(workload=workload, angles=len(idx), ref_L=ref_L, ref_ms=ref_ms, rows=rows)


def to_markdown(res) -> str:
    lines = [f"# Time-error sweep: {res['workload']}, {res['angles']} angles",
             "",
             f"Reference: sp6, FP64, {res['ref_L']} slices ({res['ref_ms']:.0f} ms). Error: "
             "max over angles of the beam-norm of the intensity difference / max reference norm.",
             "",
             "| path | integrator | dz (A) | slices | curve error | ms per curve | RHST | failed angles "
             "| CTAs per angle |",
             "|---|---|---|---|---|---|---|---|---|"]
    for r in res["rows"]:
        err = "overflow" if r["failed"] else f"{r['err']:.2e}"
        lines.append(f"| {r['precision']} | {r['integrator']} | {r['dz']:.4f} | {r['L']} | "
                     f"{err} | {r['ms']:.1f} | {r['rhst']} | {r['failed']} | {r['ctas']} |")
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="trhepd_n61", choices=sorted(W.RECIPES))
    ap.add_argument("--angles", type=int, default=60)
    ap.add_argument("--out", default="")
    ap.add_argument("--column-split", default="auto", choices=["auto", "on", "off"])
    args = ap.parse_args()
    md = to_markdown(run(args.workload, args.angles, split=args.column_split))
    if args.out:
        with open(args.out, "w") as f:
            f.write(md)
    print(md)


if __name__ == "__main__":
    main()

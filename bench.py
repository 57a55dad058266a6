"""Benchmark: rocking-curve angles/s at N = 61 beams (10 keV positrons, hexagonal 3.84 A cell,
2000 slices of 0.015 A, 60 glancing angles 0.5..6.4 deg), mixed path vs FP64 path.

One step = one pass of the whole hot path over one batch: potential tables at every kick
position (rebuilt from the device-resident structure each step), integration of all 60 angles
with the RHST, and assembly of rho and eta. Timed with CUDA events on the stream the library
launches on, after W warm-up steps; L2 (129 MB) is flushed between timed steps by writing a
256 MB buffer outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--path mixed|fp64]

Under torchrun each rank runs its own batch of angles (independent problems, no collective on
the data path); value = all ranks' angles / max over ranks of the timed seconds.
"""
from __future__ import annotations

import argparse
import json
from dataclasses import replace
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_00271_gb300 import workloads as W  # noqa: E402

METRIC = "rocking-curve angles/sec at N=61 beams: mixed vs FP64 path, <=1e-6 rel err"
UNIT = "angles/s"


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class Clocks:
    """Samples nvidia-smi every 50 ms; started before the warm-up steps (nvidia-smi takes a
    moment to start) and stopped after the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _dist():
    from paper_2306_00271_gb300 import dist as D
    return D.env()


def cpu_baseline(wl, n_angles: int):
    """The oracle (Algorithm 1 in NumPy FP64, as it stands) on a bounded sample of the angles,
    one spawn-started process per host core."""
    from oracle.curve import rocking_curve_parallel
    cores = len(os.sched_getaffinity(0))
    idx = list(np.linspace(0, len(wl.theta0) - 1, n_angles).round().astype(int))
    t = time.perf_counter()
    rocking_curve_parallel(wl, "sp4", 1000.0, angles=idx, processes=cores)
    dt = time.perf_counter() - t
    return {"value": len(idx) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(idx)} of 60 angles of the 61-beam curve (full 2000 slices each), "
                      f"{dt:.1f} s wall"}


def oracle_timings(cores: int):
    """The oracle's other timings on the host cores: O1 (conventional, eigendecomposition route)
    on the same 61-beam sample at 2000 slices and at 4000 (its Richardson level), and O1 / O2 on
    the 11-beam RHEED workload (1 angle, 400 slices)."""
    from oracle.curve import rocking_curve, rocking_curve_parallel
    out = {}
    wl = W.trhepd_n61()
    idx = list(np.linspace(0, 59, cores).round().astype(int))
    t = time.perf_counter()
    rocking_curve_parallel(wl, "conventional", angles=idx, processes=cores)
    dt = time.perf_counter() - t
    out["o1_trhepd_n61"] = {"value": len(idx) / dt, "unit": UNIT,
                            "sample": f"{len(idx)} angles, 2000 slices, {cores} processes"}
    # the second Richardson level of O1 (order 2): the same angles at half the slice width
    t = time.perf_counter()
    rocking_curve_parallel(wl.with_steps(2 * wl.n_steps), "conventional", angles=idx,
                           processes=cores)
    dt = time.perf_counter() - t
    out["o1_richardson_level_trhepd_n61"] = {
        "value": len(idx) / dt, "unit": UNIT,
        "sample": f"{len(idx)} angles, 4000 slices, {cores} processes"}
    row = W.rheed_row()
    for name, method in (("o2_rheed_row", "sp4"), ("o1_rheed_row", "conventional")):
        t = time.perf_counter()
        rocking_curve(row, method)
        out[name] = {"value": 1e6 * (time.perf_counter() - t), "unit": "us per curve",
                     "sample": "1 angle, 400 slices, 1 process"}
    return out


def rheed_row_latency():
    """Device time of one 11-beam RHEED curve (1 angle, 400 slices) per path: the small,
    latency-bound case, reported in microseconds."""
    from paper_2306_00271_gb300 import api
    wl = W.rheed_row()
    out = {}
    for path in ("fp64", "mixed"):
        eng = api.Engine(wl, path, "sp4")
        eng.rocking_curve(wl.theta0, wl.theta1)
        ms = []
        for _ in range(5):
            eng.rocking_curve(wl.theta0, wl.theta1)
            ms.append(eng.stats()["ms_integrate"])
        out[path] = {"value": 1e3 * float(np.median(ms)), "unit": "us per curve (integration)"}
        eng.close()
    return out


def run_large_sample(slices: int = 30):
    """The FP64 wide kernel on the 255-beam recipe (one structure, 120 angles) at a few slices:
    its measured time per slice-angle, the FP64 reference rate beside the mixed path's full-size
    line (at 3000 slices one FP64 curve takes about ten minutes)."""
    from paper_2306_00271_gb300 import api
    wl = W.large_n255(1)[0].with_steps(slices)
    eng = api.Engine(wl, "fp64", "sp4")
    eng.rocking_curve(wl.theta0, wl.theta1)
    ms = eng.stats()["ms_integrate"]
    tile = eng.stats()["wide_tile"]
    eng.close()
    return {"value": 120 * slices / (ms / 1e3), "unit": "angle-slices/s", "slices": slices,
            "ms": ms, "wide_tile": tile,
            "note": "FP64 wide kernel, 120 angles on 120 SMs, measured at this slice count"}


def run_large(n_sets: int = 2, slices: int = 0, n_angles: int = 0):
    """The 255-beam recipe (square 5.4 A cell, 3000 slices of 0.01 A, 120 angles 0.2..6.2 deg)
    on the mixed path for its first n_sets structures in one call: angles/s over the whole call,
    and the error of the first structure's curve against the oracle at the sampled angles of
    tests/golden/large_n255_sp4_sampled.npz (written by tests/golden/make_golden.py, which calls
    only the oracle)."""
    import torch
    from oracle.curve import curve_error
    from paper_2306_00271_gb300 import api
    sets = W.large_n255(n_sets)
    wl = sets[0].with_steps(slices) if slices else sets[0]
    if n_angles:
        wl = wl.with_angles(wl.theta0[np.linspace(0, len(wl.theta0) - 1, n_angles).astype(int)])
    eng = api.Engine(wl, "mixed", "sp4")
    eng.set_structures(np.stack([s.atoms for s in sets]))
    eng.rocking_curve(wl.theta0[:1], wl.theta1[:1])  # tables and images outside the timing
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, eta = eng.rocking_curve(wl.theta0, wl.theta1)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    st = eng.stats()
    eng.close()
    n_ang = n_sets * len(wl.theta0)
    out = {"value": n_ang / (st["ms_integrate"] / 1e3), "unit": "angles/s",
           "ms_integrate": st["ms_integrate"], "wall_s": wall, "sets": n_sets,
           "angles": n_ang, "slices": wl.n_steps, "ctas_per_angle": st["ctas_per_pair"],
           "rhst_per_angle": st["rhst_total"] / n_ang,
           "workload": "255 beams (square 5.4 A disk), %d slices of %.3f A, 120 angles "
                       "0.2..6.2 deg, sp4, mixed path, %d of the recipe's 64 structures" % (
                           wl.n_steps, -wl.z_e / wl.n_steps, n_sets)}
    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                        "large_n255_sp4_sampled.npz")
    if not slices and not n_angles and os.path.exists(gold):
        g = np.load(gold)
        e = eta.cpu().numpy()[0][g["angles"]]
        out["curve_error_vs_oracle_sampled"] = curve_error(e, g["eta"])
        out["oracle_angles"] = [int(a) for a in g["angles"]]
    return out


# DRAM bytes per kick node of the integration kernels, from one ncu capture each (dram__bytes_read
# + dram__bytes_write of a small case, divided by its node count; the traffic of these kernels is
# proportional to the node count). Summary and commands: profiles/dram_integration_trhepd_n61.md.
# Each figure holds for the kernel sources it was
# measured on: the hash of those files at capture time is stored beside it, and a figure whose
# sources have changed since is reported as null (kernel_source_hash).
KERNEL_SOURCES = {
    "mixed": ("integrate_mixed.cu", "umma.cuh", "mixed_digits.cuh", "dense_fp64.cuh", "internal.h"),
    "fp64": ("integrate_fp64.cu", "fp64_core.cuh", "internal.h"),
}
TRAFFIC_PER_NODE = {  # kernel: (bytes per node, sources, hash of the sources at capture)
    "mixed_split": ((318.562304e6 + 4.07936e6) / 2401, "mixed", "a98f9ca143e94dbb"),
    "mixed": ((320.856832e6 + 3.96544e6) / 2401, "mixed", "a98f9ca143e94dbb"),
    "fp64_split": (2.05952e6 / 361, "fp64", "07906019533b4fb9"),
    "fp64": (2.1952e6 / 361, "fp64", "07906019533b4fb9"),
}


def kernel_source_hash(group: str) -> str:
    """sha256 (16 hex digits) of the CUDA sources a kernel family is compiled from."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2306_00271_gb300",
                        "csrc")
    for name in KERNEL_SOURCES[group]:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_node(kernel: str):
    """The captured DRAM bytes per node of `kernel`, or None when its sources changed since."""
    per_node, group, captured = TRAFFIC_PER_NODE[kernel]
    return per_node if captured is not None and captured == kernel_source_hash(group) else None


# The paper's own timings (Table tab:times): another machine and another workload (Si(111)-7x7,
# 69 angles, 23 / 47 beams), quoted as context beside this run's numbers, not as its target.
PAPER_CONTEXT = {
    "source": "paper Table tab:times; Intel Core i7-12700, 8 P-cores at 2.1 GHz, oneMKL, OpenMP "
              "over angles, FP64; Si(111)-7x7 TRHEPD, 69 angles (its own workload, not this one)",
    "n23": {"orig_s": 38.306, "opt_s": 1.776, "sp4_s": 0.0381, "sp4_speedup_vs_orig": 1004,
            "sp4_angles_per_s": 1809},
    "n47": {"orig_s": 251.60, "opt_s": 8.813, "sp4_s": 0.1233, "sp4_speedup_vs_orig": 2041,
            "sp4_angles_per_s": 560},
    "note": "each row is the paper's fastest run below the conventional method's error at "
            "dz = 0.01 A; the same-machine comparison of this run is the time-error sweep "
            "(profiles/time_error_trhepd_n61.md)",
}


def algorithmic_flops(N: int, s_eff: int, L: int, n_angles: int, n_rhst_total: int) -> float:
    """Kicks: s_eff complex N x N x N products per step (8 N^3 real flops each); RHST: LU plus
    the N right-hand-side solve, (8/3 + 8) N^3 per transform."""
    return 8.0 * N ** 3 * s_eff * L * n_angles + (8.0 / 3.0 + 8.0) * N ** 3 * n_rhst_total


def run_ours(args):
    import torch
    from paper_2306_00271_gb300 import dist as D
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    D.init()
    from paper_2306_00271_gb300 import api
    wl = W.trhepd_n61()
    if args.slices:
        wl = wl.with_steps(args.slices)
    A = len(wl.theta0)
    dev = torch.device("cuda", local)
    engines = {}
    for path in args.paths:
        engines[path] = api.Engine(wl, path, "sp4")
        engines[path].set_column_split(args.column_split)
    atoms_d = torch.tensor(wl.atoms, dtype=torch.float64, device=dev)
    dw_d = torch.tensor(wl.dw, dtype=torch.float64, device=dev)
    t0_d = torch.tensor(wl.theta0, dtype=torch.float64, device=dev)
    t1_d = torch.tensor(wl.theta1, dtype=torch.float64, device=dev)
    rho = torch.empty((1, A, wl.n_beams), dtype=torch.complex128, device=dev)
    eta = torch.empty((1, A, wl.n_beams), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    results = {}
    for path, eng in engines.items():
        def step():
            eng.set_structures(atoms_d, dw_d)
            eng.rocking_curve(t0_d, t1_d, rho, eta)
            return eng.stats()
        clocks = Clocks(local)
        clocks.start()
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        ms_steps, ms_int, ms_pot, launches, rhst, split = [], [], [], 0, 0, 0
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            ev0.record()
            st = step()
            ev1.record()
            torch.cuda.synchronize()
            ms_steps.append(ev0.elapsed_time(ev1))
            ms_int.append(st["ms_integrate"])
            ms_pot.append(st["ms_potential"])
            launches += st["kernels_launched"]
            rhst += st["rhst_total"]
            split = st["column_split"]
        clk = clocks.stop()
        total_ms = float(np.sum(ms_steps))
        total_ms = D.max_over_ranks(total_ms)
        # end to end through the public API with host buffers: H2D of the step's inputs and
        # D2H of its outputs inside the timed region
        # (asynchronous calls into pinned host buffers: the steps queue back to back and the
        # host waits once, after the last; every step's copies are inside the timed region)
        atoms_h = np.ascontiguousarray(wl.atoms)
        dw_h = np.ascontiguousarray(wl.dw)
        rho_t = torch.empty((1, A, wl.n_beams), dtype=torch.complex128, pin_memory=True)
        eta_t = torch.empty((1, A, wl.n_beams), dtype=torch.float64, pin_memory=True)
        rho_h, eta_h = rho_t.numpy(), eta_t.numpy()
        e2e_steps = max(10, args.steps)
        eng.set_async(True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(e2e_steps):
            eng.set_structures(atoms_h, dw_h)
            eng.rocking_curve_host(wl.theta0, wl.theta1, rho_h, eta_h)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t) / e2e_steps
        e2e_bad = eng.stats()["n_bad"]
        eng.set_async(False)
        results[path] = dict(ms_per_step=total_ms / args.steps, ms_integrate=float(np.mean(ms_int)),
                             ms_potential=float(np.mean(ms_pot)), launches=launches,
                             rhst_per_step=rhst / args.steps, clocks=clk, column_split=split,
                             value=ws * A * args.steps / (total_ms / 1e3),
                             e2e=dict(value=ws * A / e2e_s, unit=UNIT, steps=e2e_steps,
                                      n_bad=e2e_bad, mode="asynchronous calls, pinned host "
                                      "buffers, one wait after the last step",
                                      h2d_bytes_per_step=int(atoms_h.nbytes + dw_h.nbytes
                                                             + 2 * A * 8),
                                      d2h_bytes_per_step=int(rho_h.nbytes + eta_h.nbytes)),
                             eta=eta.detach().cpu().numpy()[0].copy())
    return wl, results, ws, rank


def run_gradient(local: int, slices: int = 0, warmup: int = 1, path: str = "fp64"):
    """One R-factor gradient at the differentiation workload (N = 61, 2000 slices, 60 angles,
    12 free z + 6 Debye-Waller classes, checkpoints every 64 steps): binary64 recompute and
    adjoint, the contraction in binary64 (FP64 context) or as BF16 digit products (mixed). The
    target curve is this library's own FP64 curve at the hidden true structure."""
    import torch
    from paper_2306_00271_gb300 import api
    fp = W.rfactor_fit()
    if slices:
        fp = replace(fp, workload=fp.workload.with_steps(slices))
    wl = fp.workload
    eng = api.Engine(wl, path, "sp4")
    truth = W.fit_structure(fp, fp.z_true, fp.b_true)
    eng.set_structures(truth.atoms[None], truth.dw[None])
    _, eta_t = eng.rocking_curve(wl.theta0, wl.theta1)
    target = eta_t[0, :, 0].contiguous()
    eng.set_structures(wl.atoms[None], wl.dw[None])
    eng.set_fit(fp.free_atoms, fp.dw_class, ckpt_every=64)
    for _ in range(warmup):
        eng.rfactor_grad(wl.theta0, wl.theta1, target)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    R, gz, gb = eng.rfactor_grad(wl.theta0, wl.theta1, target)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = eng.stats()
    eng.close()
    return {"metric": f"R-factor gradients/s (N=61, L={wl.n_steps}, 60 angles, 18 parameters, "
                      + ("mixed forward, reverse sweep binary64 with the contraction on BF16 "
                         "digits, " if path == "mixed" else "FP64 forward, FP64 reverse sweep, ")
                      + "checkpoints every 64 steps)",
            "value": 1000.0 / ms, "unit": "gradients/s", "ms_per_gradient": ms,
            "ms_forward": st["ms_integrate"], "ms_reverse": st["ms_gradient"],
            "kernels_launched": st["kernels_launched"], "R": float(R[0])}


def run_gradient_large(slices: int = 30, n_angles: int = 16):
    """The 255-beam recipe's gradient on a stated sample: its first structure, n_angles of its
    120 angles, the first `slices` slices of 0.01 A (a slab of slices * 0.01 A; the full 3000
    would take the binary64 sweep tens of minutes), the z of its 8 surface atoms and 4
    Debye-Waller classes of 2 of them as the 12 parameters, one checkpoint segment. Reports the
    measured gradient time and its rate in angle-slices/s (not extrapolated)."""
    import torch
    from paper_2306_00271_gb300 import api
    wl = W.large_n255(1)[0]
    wl = replace(wl, z_e=-0.01 * slices).with_steps(slices)
    wl = wl.with_angles(wl.theta0[np.linspace(0, len(wl.theta0) - 1, n_angles).astype(int)])
    free = np.arange(8)
    cls = np.full(wl.atoms.shape[0], -1)
    cls[:8] = np.arange(8) // 2
    eng = api.Engine(wl, "fp64", "sp4")
    eng.set_fit(free, cls, ckpt_every=slices)
    target = np.full(n_angles, 1.0 / n_angles)
    eng.rfactor_grad(wl.theta0, wl.theta1, target)   # tables, tuner probe
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    R, gz, gb = eng.rfactor_grad(wl.theta0, wl.theta1, target)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = eng.stats()
    eng.close()
    return {"metric": "R-factor gradient, 255 beams (wide binary64 reverse sweep), 12 parameters",
            "value": 1000.0 / ms, "unit": "gradients/s", "ms_per_gradient": ms,
            "ms_forward": st["ms_integrate"], "ms_reverse": st["ms_gradient"],
            "angle_slices_per_s": n_angles * slices / (ms / 1e3), "angles": n_angles,
            "slices": slices, "sample": f"{n_angles} of 120 angles, first {slices} of 3000 "
                                        "slices of 0.01 A, 1 of 64 structures",
            "wide_tile": st["wide_tile"], "R": float(R[0])}


def run_batches(slices: int = 0):
    """A small batched line: 8 perturbed structures (4 with 31 and 4 with 61 beams) x 60 angles
    on the mixed path at 2000 slices, one persistent launch replayed from its CUDA graph, timed
    with CUDA events around the replay (after one eager run that also captures the graph); the
    per-curve error of each batched curve against the FP64 GPU path is reported beside it."""
    import torch
    from oracle.curve import curve_error
    from paper_2306_00271_gb300 import api
    sets = W.batch_sets(12)
    classes = {31: [], 61: []}
    for s_ in sets:
        n = s_.beams.shape[0]
        if n in classes and len(classes[n]) < 4:
            classes[n].append(s_)
    L = slices or 2000
    batch = api.Batch()
    engines, outs, n_angles = {}, {}, 0
    for n, members in classes.items():
        wl = members[0].with_steps(L)
        eng = api.Engine(wl, "mixed", "sp4")
        eng.set_structures(np.stack([m.atoms for m in members]))
        outs[n] = batch.add(eng, wl.theta0, wl.theta1)
        engines[n] = (eng, wl, members)
        n_angles += len(members) * len(wl.theta0)
    batch.run()                      # eager run + capture
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    batch.run()                      # graph replay
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = batch.stats()
    errs = []
    for n, (eng, wl, members) in engines.items():
        ref = api.Engine(wl, "fp64", "sp4")
        ref.set_structures(np.stack([m.atoms for m in members]))
        _, eta_f = ref.rocking_curve(wl.theta0, wl.theta1)
        eta_b = outs[n][1].cpu().numpy()
        eta_f = eta_f.cpu().numpy()
        errs += [curve_error(eta_b[k], eta_f[k]) for k in range(len(members))]
        ref.close()
    out = {"mixed": {"value": n_angles / (ms / 1e3), "unit": "angles/s", "ms": ms,
                     "angles": n_angles, "slices": L, "path": "mixed",
                     "beam_classes": {str(n): len(m[2]) for n, m in engines.items()},
                     "graph_replay": st["graph_replay"], "launches": st["kernels_launched"],
                     "per_curve_error_vs_fp64_gpu": {"max": float(np.max(errs)),
                                                     "median": float(np.median(errs)),
                                                     "curves": len(errs)}}}
    batch.close()
    for eng, _, _ in engines.values():
        eng.close()
    return out


def run_wide_121(slices: int = 0):
    """One 121-beam structure of the batched workload (set 2: 10 keV positrons, hexagonal 3.84 A,
    2000 slices, 60 angles) on the mixed path (a 4-CTA cluster per angle) and on the FP64 wide
    kernel at the same full depth: angles/s of each and the curve error between them."""
    import torch
    from oracle.curve import curve_error
    from paper_2306_00271_gb300 import api
    wl = [s for s in W.batch_sets(3) if s.beams.shape[0] == 121][0]
    if slices:
        wl = wl.with_steps(slices)
    out, etas = {}, {}
    for path in ("mixed", "fp64"):
        # one call each (the FP64 curve takes half a minute): the library's own CUDA events
        # around its integration launches (mixed: the cluster kernel and the assembly), the
        # potential tables and digit images outside them
        eng = api.Engine(wl, path, "sp4")
        _, eta = eng.rocking_curve(wl.theta0, wl.theta1)
        torch.cuda.synchronize()
        st = eng.stats()
        ms = st["ms_integrate"]
        etas[path] = eta.cpu().numpy()[0]
        out[path] = {"value": len(wl.theta0) / (ms / 1e3), "unit": "angles/s", "ms": ms,
                     "ms_tables": st["ms_potential"], "ctas_per_angle": st["ctas_per_pair"],
                     "rhst_per_curve": st["rhst_total"]}
        eng.close()
    out["mixed_vs_fp64_curve_error"] = curve_error(etas["mixed"], etas["fp64"])
    out["speedup_mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["workload"] = (f"121 beams (hexagonal shell), {wl.n_steps} slices of "
                       f"{-wl.z_e / wl.n_steps:.3f} A, 60 angles 0.5..6.4 deg, sp4")
    out["_eta_fp64"] = etas["fp64"]
    return out


def run_config2(n_sets: int = 512, slices: int = 0, eta_121_fp64=None, oracle_angles=(7, 41)):
    """The batching + precision recipe at its stated size: 512 parameter sets (surface z of the
    61-beam structure perturbed by N(0, 0.3^2) A, seeds 3000 + k), beam counts 31 / 61 / 121 round
    robin, 60 angles each, 2000 slices, all on the mixed path in one batch: the three beam
    classes as three jobs, their sets in chunks whose digit images fit the image budget, every
    chunk's image builds and launches in one captured launch sequence. The timed run is the
    batch's eager run (the same kernels the graph replays; the graph itself is captured during
    it without running). Per-curve errors: every curve of the first set of each class against
    the FP64 GPU path (all 60 angles), and two sampled angles of those sets against the oracle."""
    import torch
    from oracle.curve import curve_error, rocking_curve_parallel
    from paper_2306_00271_gb300 import api
    sets = W.batch_sets(n_sets)
    L = slices or 2000
    classes = {}
    for s_ in sets:
        classes.setdefault(s_.beams.shape[0], []).append(s_)
    batch = api.Batch()
    jobs = {}
    for n in sorted(classes):
        members = classes[n]
        wl = members[0].with_steps(L)
        eng = api.Engine(wl, "mixed", "sp4")
        eng.set_image_budget(96 << 30)
        eng.set_structures(np.stack([m.atoms for m in members]))
        rho, eta = batch.add(eng, wl.theta0, wl.theta1)
        jobs[n] = (eng, wl, members, eta)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t = time.perf_counter()
    ev0.record()
    batch.run()
    ev1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t
    ms = ev0.elapsed_time(ev1)
    st = batch.stats()
    n_angles = sum(len(j[2]) * len(j[1].theta0) for j in jobs.values())
    per_class = {}
    for n, (eng, wl, members, eta) in jobs.items():
        e_mixed = eta[0].cpu().numpy()
        if n == 121 and eta_121_fp64 is not None and L == 2000:
            e_ref = eta_121_fp64
        else:
            ref = api.Engine(members[0].with_steps(L), "fp64", "sp4")
            _, e_ref = ref.rocking_curve(wl.theta0, wl.theta1)
            e_ref = e_ref.cpu().numpy()[0]
            ref.close()
        rec = {"sets": len(members), "curve_error_vs_fp64_gpu_set0": curve_error(e_mixed, e_ref)}
        if oracle_angles:
            _, eta_o, _, _ = rocking_curve_parallel(members[0].with_steps(L), "sp4",
                                                    angles=list(oracle_angles),
                                                    processes=len(oracle_angles))
            rec["error_vs_oracle_set0_sampled_angles"] = curve_error(
                e_mixed[list(oracle_angles)], eta_o)
            rec["oracle_angles"] = list(oracle_angles)
        per_class[str(n)] = rec
    out = {"value": n_angles / (ms / 1e3), "unit": "angles/s", "ms": ms, "wall_s": wall,
           "sets": n_sets, "angles": n_angles, "slices": L, "path": "mixed",
           "set_chunks": st["set_chunks"], "launches": st["kernels_launched"],
           "per_class": per_class,
           "note": "timed run = the batch's eager run; errors: eacc-style curve error, FP64 GPU "
                   "path on all 60 angles of each class's first set, oracle on two angles"}
    batch.close()
    for j in jobs.values():
        j[0].close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="auto", choices=["auto", "mixed", "fp64"])
    ap.add_argument("--cpu-angles", type=int, default=0)
    ap.add_argument("--slices", type=int, default=0,
                    help="override the slice count (small cases for profiling; not a bench line)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle timing")
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload lines")
    ap.add_argument("--no-config2", action="store_true",
                    help="skip the 512-set batching + precision recipe")
    ap.add_argument("--config2-sets", type=int, default=512,
                    help="parameter sets of the batching recipe (512 = its stated size)")
    ap.add_argument("--column-split", default="auto", choices=["auto", "on", "off"],
                    help="two CTAs per angle (auto: the autotuner times both forms on probes "
                         "of the call and keeps the faster)")
    ap.add_argument("--large-only", action="store_true",
                    help="only the 255-beam mixed line (profiling cases with --slices and "
                         "--large-angles; not the bench line)")
    ap.add_argument("--large-sets", type=int, default=2)
    ap.add_argument("--large-angles", type=int, default=0)
    ap.add_argument("--grad-only", default=None, choices=["mixed", "fp64"],
                    help="only the 18-parameter gradient line on a context of this precision "
                         "(one warm-up gradient, one timed; profiling runs, not the bench line)")
    args = ap.parse_args()
    ws, rank, _ = _dist()
    if args.large_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_large(args.large_sets, args.slices, args.large_angles)))
        return
    if args.grad_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(run_gradient(0, args.slices, path=args.grad_only)))
        return
    wl = W.trhepd_n61()
    cfg = {"workload": "trhepd_n61: 10 keV e+, hex a=3.84 A, N=61 beams, 16 atoms, "
                       "L=2000 x 0.015 A, 60 angles 0.5..6.4 deg, sp4, RHST threshold 1000",
           "n_beams": 61, "n_steps": 2000, "n_angles": 60, "integrator": "sp4",
           "l2": "flushed between timed steps (256 MB write outside the events)",
           "parallelism": f"replicas x{ws}"}
    if args.impl == "reference":
        if rank != 0:
            return
        # W untimed and K timed steps, each the oracle on a bounded sample of the workload's
        # angles (one process per host core)
        n = args.cpu_angles or min(60, max(8, len(os.sched_getaffinity(0))))
        for _ in range(args.warmup):
            cpu_baseline(wl, n)
        runs = [cpu_baseline(wl, n) for _ in range(max(1, args.steps))]
        secs = sum(n / r["value"] for r in runs)
        value = n * len(runs) / secs
        cb = dict(runs[-1], value=value,
                  sample=f"{n} of 60 angles of the 61-beam curve (full 2000 slices each) per "
                         f"step, {len(runs)} timed steps, {secs:.1f} s wall")
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": value,
                          "unit": UNIT, "n_gpus": args.gpus, "steps": len(runs),
                          "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(runs),
                          "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": cfg, "cpu_baseline": cb,
                          "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return
    from paper_2306_00271_gb300 import api
    paths = ["fp64"] if args.path == "fp64" else (["mixed"] if args.path == "mixed" else [])
    if args.path == "auto":
        paths = ["fp64"]
        try:
            api.Engine(wl, "mixed", "sp4").close()
            paths = ["mixed", "fp64"]
        except api.TrhError:
            pass
    args.paths = paths
    wl, res, ws, rank = run_ours(args)
    if rank != 0:
        return
    if args.slices:
        cfg["n_steps"] = wl.n_steps
        cfg["workload"] = cfg["workload"].replace("L=2000", f"L={wl.n_steps}") + " (profiling case)"
    head = res[paths[0]]
    peaks = _peaks() or {}
    N, L, A = 61, wl.n_steps, len(wl.theta0)
    flops = algorithmic_flops(N, 6, L, A, int(round(head["rhst_per_step"])))
    achieved = flops / (head["ms_integrate"] / 1e3) / 1e12
    if paths[0] == "mixed":
        peak = peaks.get("bf16_tflops", 1900.0)
        kern = "mixed_split" if head["column_split"] else "mixed"
        tpn = traffic_per_node(kern)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": None if tpn is None else tpn * (6 * L + 1),
                "peak_source": "MEASURED_PEAKS.json bf16 burst (of measured)",
                "note": "achieved counts complex FP32-equivalent algorithmic flops",
                # each algorithmic product costs ten BF16 digit products (four digits per
                # operand, orders 0..3), so the tensor pipe's own ceiling for this arithmetic
                # is a tenth of the BF16 peak
                "digit_product_ceiling": peak / 10.0,
                "frac_of_digit_product_ceiling": achieved / (peak / 10.0)}
    else:
        bf = peaks.get("bf16_tflops", 1900.0)
        peak = bf * 1.25 / 2250.0
        tpn = traffic_per_node("fp64_split" if head["column_split"] else "fp64")
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": None if tpn is None else tpn * (6 * L + 1),
                "peak_source": "fp64: measured bf16 burst x nominal fp64/bf16 ratio (1.25/2250); "
                               "DMMA microbenchmark on this pool: 1.05 TFLOP/s"}
    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16x4+f32pair" if paths[0] == "mixed" else "f64",
           "data": "synthetic (seeded structure, see paper_2306_00271_gb300/workloads.py)",
           "config": dict(cfg, path=paths[0],
                          ctas_per_angle=2 if head.get("column_split") else 1),
           "e2e": head["e2e"],
           "gpu_launches": int(head["launches"]), "clocks": head["clocks"],
           "roofline": roof,
           "kernels_ms": {"integrate": head["ms_integrate"], "potential": head["ms_potential"]},
           "rhst_per_curve": head["rhst_per_step"]}
    for p in paths[1:]:
        out[f"{p}_path"] = {"value": res[p]["value"], "ms_per_step": res[p]["ms_per_step"],
                            "ms_integrate": res[p]["ms_integrate"]}
    if "mixed" in res and "fp64" in res:
        from oracle.curve import curve_error
        out["mixed_vs_fp64_curve_error"] = curve_error(res["mixed"]["eta"], res["fp64"]["eta"])
    if not args.no_grad:
        out["gradient"] = run_gradient(int(os.environ.get("LOCAL_RANK", "0")), args.slices)
        out["gradient_mixed_forward"] = run_gradient(int(os.environ.get("LOCAL_RANK", "0")),
                                                     args.slices, path="mixed")
    if not args.no_batch:
        out["batches"] = run_batches(args.slices)
        wide = run_wide_121(args.slices)
        eta_ref = wide.pop("_eta_fp64")
        out["wide_121"] = wide
        if not args.no_config2:
            out["config2_full"] = run_config2(args.config2_sets, args.slices,
                                              eta_121_fp64=eta_ref)
        out["large_n255"] = run_large(2, args.slices)
        out["large_n255_fp64_sample"] = run_large_sample()
        if not args.no_grad:
            out["large_n255_gradient_sample"] = run_gradient_large()
        out["rheed_row_latency"] = rheed_row_latency()
    out["paper_context"] = PAPER_CONTEXT
    if ws == 1 and not args.no_cpu:
        n = args.cpu_angles or min(60, max(8, len(os.sched_getaffinity(0))))
        try:
            out["cpu_baseline"] = cpu_baseline(wl, n)
            out["oracle_timings"] = oracle_timings(len(os.sched_getaffinity(0)))
        except Exception as e:  # pragma: no cover
            out["cpu_baseline"] = {"error": str(e)}
    print(json.dumps(out))


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Throughput of the (X)MS-CASPT2 amplitude / effective-Hamiltonian path on GB300.

One step = one caspt2_solve + caspt2_densities of the synthetic benzophenone-like
XMS-CASPT2 workload (nclosed 20, nact 8 with 8 electrons, nvirt 200, naux 700, 3 states,
shift 0.2, MS-MR): setup (SA density, mean field, core energy, XMS rotation, rotated
RDMs, H^ref), the amplitude solves of all eight classes, H^eff and its eigenpairs, lambda
of state 0, and the densities d1, d2 and D1 in DF form of state 0.  Inputs are resident
in HBM before the timed region; L2 is flushed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own copy of the
workload (independent solves, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amp+λ solves/s & TFLOP/s vs FP64 GPU form at |ΔE|≤1e-8 Eh; serve p50/p99 ms"
WORKLOAD = "c20a8v200x700n3"
OPTS = dict(xms=1, scheme=0, shift=0.2)
WORKLOAD_DESC = ("XMS-CASPT2 MS-MR, nclosed 20, nact 8 (8e, 4900 dets), nvirt 200, naux 700, "
                 "3 states, shift 0.2 Eh, seed 1 (benzophenone-like synthetic)")
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (no measured FP64 peak is provided)
# dram__bytes_read.sum + dram__bytes_write.sum of one k_classH launch at this workload
# (ncu capture summarised in profiles/); None until captured for the current kernel.
CLASSH_TRAFFIC_BYTES = None


def classh_flops(c, v, X):
    """Algorithmic flops of the class-H DF contraction: K_ij^ab = sum_P B_Pai B_Pbj for
    i <= j and all (a, b) (K_ji is K_ij transposed), 2 flops per multiply-add."""
    return 2.0 * (c * (c + 1) / 2) * v * v * X


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device, self.proc = device, None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[2 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs():
    from synth import make_problem, WORKLOADS
    return make_problem(**WORKLOADS[WORKLOAD], kmax=4)


def oracle_solve(p):
    """The CPU oracle for the same step (setup, classes A-H, H^eff, lambda of state 0)."""
    from oracle import o2_rdm as o2
    from oracle import o2_classes as oc
    st = o2.setup(p, xms=bool(OPTS["xms"]), kmax=4)
    mom = oc.all_moments(p, st, shift=OPTS["shift"], scheme="msmr")
    parts = {c: (-np.einsum("llk->lk", M1), np.diagonal(M2).copy()) for c, (M1, M2, M3) in mom.items()}
    H, w, R = o2.heff(st, parts, OPTS["shift"])
    lam = {c: oc.lambda_pieces(*mom[c], R, 0, OPTS["shift"]) for c in mom}
    return H, w, R, lam


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def time_oracle(p, budget_s=20.0, max_runs=3):
    """Time the oracle on the host cores for a bounded sample (whole solves)."""
    ts, last = [], None
    t_all = time.perf_counter()
    while len(ts) < max_runs and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        last = oracle_solve(p)
        ts.append(time.perf_counter() - t0)
    return ts, last


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    p = make_inputs()
    for _ in range(args.warmup):
        oracle_solve(p)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve(p)
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "classes": "ABCDEFGH", "form": "oracle (numpy FP64)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(),
                         "kind": "oracle",
                         "sample": (f"{args.steps} whole amplitude + lambda solves of the workload "
                                    "(densities not included: the oracle's density pass alone "
                                    "takes about 190 s on 8 cores)")},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import paper_1606_01273_gb300 as cp

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    cp.lib()

    p = make_inputs()
    host = cp.problem_inputs(p)
    h2d = sum(x.nbytes for x in host if x is not None)
    n = p.nstate
    # energies, per-class pieces and lambda, plus d1 and d2 (GDF stays in HBM for the
    # gradient contraction with the derivative integrals)
    d2h = 8 * (4 * n * n + 2 * n + 1 + 8 * (n * n + n)) + 2 * 8 * p.nmo * p.nmo
    dev_in = [torch.from_numpy(x).to(dev) for x in host]   # f, B, rdm1-4
    popt = dict(OPTS, precision=cp.BF16X if args.precision == "bf16x" else cp.FP64,
                slices=args.slices)
    ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **popt)
    ctx.set_inputs(*dev_in)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            ctx.solve(stream.cuda_stream)
            ctx.compute_densities(stream=stream.cuda_stream)
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kern_ms, launches, tri, dens_ms = [], 0, [], []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))                # L2 flush outside the timed events
                ev[k][0].record(stream)
                ctx.solve(stream.cuda_stream)
                ctx.compute_densities(stream=stream.cuda_stream)
                ev[k][1].record(stream)
            r = ctx.result()
            dens_ms.append(r.timings_ms[8])
            kern_ms.append(r.timings_ms[4])
            tri.append((r.timings_ms[5], r.timings_ms[6], r.timings_ms[7]))
            launches += r.launches
        torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if ws > 1:
        t = torch.tensor([total_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    value = ws * args.steps / total_s
    last = ctx.result()

    # end to end through the C ABI with host buffers (pinned), H2D + D2H inside the timing
    pinned = [torch.from_numpy(x).pin_memory() for x in host]
    ctx_h = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **popt)
    for _ in range(max(1, args.warmup)):
        ctx_h.set_inputs(*pinned)
        ctx_h.solve()
        ctx_h.compute_densities()
        ctx_h.result()
        ctx_h.get_densities(with_gdf=False)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx_h.set_inputs(*pinned)
        ctx_h.solve()
        ctx_h.compute_densities()
        ctx_h.result()
        ctx_h.get_densities(with_gdf=False)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = ws * args.steps / e2e_s
    ctx_h.close()

    if rank != 0:
        ctx.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    kavg = statistics.mean(kern_ms)
    flops = classh_flops(p.nclosed, p.nvirt, p.naux)
    achieved = flops / (kavg * 1e-3) / 1e12
    tri_ms = sum(t[0] for t in tri)
    tri_fl = sum(t[1] for t in tri)
    tri_n = sum(t[2] for t in tri)
    tri_avg_ms = tri_ms / max(tri_n, 1)
    tri_achieved = tri_fl / max(tri_ms * 1e-3, 1e-12) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "classes": cp.supported_classes(),
                   "form": "plain FP64", "parallelism": f"{ws} independent solve(s)",
                   "l2": "256 MB write between steps; B (291 MB) larger than L2"},
        "tflops_classH_kernel": achieved,
        # dominant kernel by device time (see profiles/): the Householder tridiagonalisation
        # of the class overlap / Fock matrices; FP64, 4/3 m^3 algorithmic flops per launch
        "roofline": {"bound": "alu", "achieved": tri_achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": tri_achieved / FP64_PEAK_TFLOPS,
                     "traffic": None, "kernel": "k_tridiag", "kernel_ms": tri_avg_ms,
                     "launches_per_step": tri_n / max(len(tri), 1),
                     "flops_per_launch": tri_fl / max(tri_n, 1),
                     "peak_kind": "nominal FP64 (no measured FP64 peak in MEASURED_PEAKS)"},
        "roofline_classH": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                            "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                            "traffic": CLASSH_TRAFFIC_BYTES, "kernel": "k_classH",
                            "kernel_ms": kavg, "flops_per_launch": flops},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "stage_ms_last": dict(zip(["setup", "classH", "classesAG", "heff_lambda", "classH_kernel",
                                   "tridiag_kernel_total"], last.timings_ms[:6]),
                              densities=statistics.mean(dens_ms)),
    }
    if ws == 1 and not args.no_cpu_baseline:
        ts, ref = time_oracle(p)
        w = ref[1]
        line["cpu_baseline"] = {"value": len(ts) / sum(ts), "unit": "solves/s",
                                "cores": cpu_cores(), "kind": "oracle",
                                "sample": (f"{len(ts)} whole amplitude + lambda solve(s) of the "
                                           "workload (setup, classes A-H, H^eff, lambda), numpy "
                                           "FP64; the oracle's density pass is not in the sample "
                                           "(about 190 s on 8 cores), so this rate is an upper "
                                           "bound for the oracle's full step")}
        line["parity"] = {"max_abs_dE_Eh": float(np.abs(last.Ems - w).max()), "tol_Eh": 1e-8}
    print(json.dumps(line))
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "bf16x"], default="fp64")
    ap.add_argument("--slices", type=int, default=7)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

#!/usr/bin/env python
"""Throughput of the (X)MS-CASPT2 amplitude / lambda path on GB300.

Default workload: the synthetic copper-corrole shape (nclosed 70, nact 10 with 10
electrons, nvirt 600, naux 2000, 5 states, XMS, MS-MR, vertical shift 0.3 Eh, DF decay
sigma_k = exp(-k/40)).  One step = one caspt2_solve: setup (SA density, mean field, core
energy, XMS rotation, rotated 1-4-RDMs, H^ref), the amplitude solves of all eight classes,
H^eff and its eigenpairs, and lambda of state 0 (the metric's "amp + lambda" solve).  The
densities are not in this workload's step: their all-tuple amplitude arrays of class G
alone would need about 250 GB.  `--workload c20a8v200x700n3` times the smaller XMS
workload (nclosed 20, nact 8, nvirt 200, naux 700, 3 states, shift 0.2) with the
densities of state 0 in the step.  Inputs are resident in HBM before the timed region; L2
is flushed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]

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
BENCH = {
    "c70a10v600x2000n5": dict(
        opts=dict(xms=1, scheme=0, shift=0.3), densities=False,
        desc=("XMS-CASPT2 MS-MR, nclosed 70, nact 10 (10e, 63504 dets), nvirt 600, naux 2000, "
              "5 states, shift 0.3 Eh, sigma_k = exp(-k/40), seed 4 (copper-corrole-shaped "
              "synthetic)"),
        step="caspt2_solve: setup, amplitudes of classes A-H, H^eff, E_MS, lambda of state 0"),
    "c42a12v350x1200n4": dict(
        opts=dict(xms=1, scheme=0, shift=0.2), densities=False,
        desc=("XMS-CASPT2 MS-MR, nclosed 42, nact 12 (12e, 853776 dets), nvirt 350, naux 1200, "
              "4 states, shift 0.2 Eh, seed 3 (benzophenone-shaped synthetic)"),
        step="caspt2_solve: setup, amplitudes of classes A-H, H^eff, E_MS, lambda of state 0"),
    "c20a8v200x700n3": dict(
        opts=dict(xms=1, scheme=0, shift=0.2), densities=True,
        desc=("XMS-CASPT2 MS-MR, nclosed 20, nact 8 (8e, 4900 dets), nvirt 200, naux 700, "
              "3 states, shift 0.2 Eh, seed 1"),
        step="caspt2_solve + caspt2_densities (d1, d2, D1 in DF form of state 0)"),
}
DEFAULT_WORKLOAD = "c70a10v600x2000n5"
WORKLOAD = DEFAULT_WORKLOAD
OPTS = BENCH[WORKLOAD]["opts"]
WORKLOAD_DESC = BENCH[WORKLOAD]["desc"]
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (no measured FP64 peak is provided)
# dram__bytes_read.sum + dram__bytes_write.sum of one k_classH launch at this workload
# (ncu capture summarised in profiles/); None until captured for the current kernel.
CLASSH_TRAFFIC_BYTES = None
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) from ncu captures of the current
# kernels on this workload (bench.py --profile-case classA / classH):
#   k_tridiag_smem, m = 1536: 18.94 MB + 14.08 MB against 28.31 MB algorithmic
#   k_oz_gemm, class-H K = Bcv^T Bcv (4000 x 4000 x 700, 7 slices): 45.89 MB + 85.85 MB
TRIDIAG_DRAM_PER_ALG_BYTE = (18.944512e6 + 14.080000e6) / (8.0 * 1536 ** 2 + 4.0 * 1536 * 1535)
CLASSH_SPLIT_TRAFFIC_BYTES = 45.892096e6 + 85.852416e6


def measured_peak(key, fallback):
    """(peak, kind): a peak from MEASURED_PEAKS.json (measured on this machine), else the stated
    fallback (one earlier GB300 measurement)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key]), "measured (MEASURED_PEAKS.json %s)" % key
    except (OSError, KeyError, ValueError, TypeError):
        return fallback, "fallback (MEASURED_PEAKS.json absent on this machine)"


def classh_flops(c, v, X):
    """Algorithmic flops of the class-H DF contraction: K_ij^ab = sum_P B_Pai B_Pbj for
    i <= j and all (a, b) (K_ji is K_ij transposed), 2 flops per multiply-add."""
    return 2.0 * (c * (c + 1) / 2) * v * v * X


def dist_env():
    from paper_1606_01273_gb300.shard import dist_env as env
    return env()


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


def make_inputs(kmax=4):
    from synth import make_problem, WORKLOADS
    return make_problem(**WORKLOADS[WORKLOAD], kmax=kmax)


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


def solve_flops(c, a, v, X, n):
    """Algorithmic FP64-equivalent flops of one MS-MR solve: the class-H pair integrals
    (2 (cv)^2 X, both (i, j) orders), the DF integral blocks of the other classes' sources
    (one GEMM of 2 X over each block's index pairs), the two m^3-type eigensolves and the
    X^T F X transforms of every sector (4/3 m^3 + 4/3 m^3 + 3 * 2 m^3 per sector, m the
    sector dimension), and the sector transforms of the sources (2 m * tuples * n per
    sector)."""
    cv = c * v
    fl = 2.0 * cv * cv * X
    # integral blocks (pq|rt) used by the sources of classes A-G
    for n0, n1 in ((v * a, v * c), (v * a, v * a), (c * a, c * a), (v * c, a * a), (v * a, c * a)):
        fl += 2.0 * n0 * n1 * X
    sectors = {"A": (a ** 3 * n, c), "C": (a ** 3 * n, v), "D": (2 * a * a * n, c * v),
               "B": (a * a * n, c * c), "F": (a * a * n, v * v), "E": (a * n, v * c * c),
               "G": (a * n, v * v * c)}
    for m, ntup in sectors.values():
        fl += (4.0 / 3.0 + 4.0 / 3.0 + 6.0) * m ** 3 + 2.0 * m * ntup * n
    return fl


def classh_sample(p, nclosed_sample=2):
    """Bounded oracle sample for large workloads: the oracle's class-H moment sums over the
    first group of `nclosed_sample` closed orbitals (rows i of K(ai|bj) against every j),
    timed on the host cores.  Returns (seconds, fraction of the solve's algorithmic flops
    that the sample covers)."""
    from oracle import o2_rdm as o2
    st = o2.setup(p, xms=bool(OPTS["xms"]), kmax=2)
    t0 = time.perf_counter()
    o2.class_h_moments(p, st, shift=OPTS["shift"], scheme="msmr", i_chunk=nclosed_sample,
                       i_groups=1)
    dt = time.perf_counter() - t0
    c, a, v, X = p.nclosed, p.nact, p.nvirt, p.naux
    frac = (2.0 * nclosed_sample * v * c * v * X) / solve_flops(c, a, v, X, p.nstate)
    return dt, frac


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", name + ".json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except OSError:
        return None


def conditioning_bound(g, shift, dw=1e-14):
    """First-order bound on |dE_MS| from an error dw in every sector eigenvalue omega:
    d<Psi1_L|H|L~>/d omega = sum V^2/D^2 = norm_L and d<Psi1_L|Psi1_L>/d omega =
    -2 sum V^2/D^3 = -2 M3_L, so |dH^eff_LL| <= dw (norm_L + 2 E_s |M3_L|) summed over the
    classes (taken over the states: E_MS mixes them through R)."""
    b = 0.0
    for L in range(len(g["Ems"])):
        s = sum(g["norm_class"][c][L] + 2.0 * shift * abs(g["M3"][c][L]) for c in g["norm_class"])
        b = max(b, dw * s)
    return b


SERVE_DESC = ("256 Poisson arrivals (mean 20/s, at most 16 outstanding) of XMS-CASPT2 "
              "requests (MS-MR, shift 0.2, all classes, target-state densities for every other "
              "request) drawn from 12 "
              "synthetic problems with sizes uniform over nclosed 4-42, nact 4-8, nvirt "
              "20-350, 1-4 states, naux = 3 nmo (the serving-stream size range with nact "
              "capped at 8: a 12-orbital request carries a 55 GB 4-RDM)")


def serve_problems(count=12, seed=5000):
    """The serving pool: distinct seeded problems of mixed size (inputs only), sizes uniform
    over nclosed 4-42, nact 4-8, nvirt 20-350, 1-4 states (CASCI, RDMs and the DF factor
    product on the GPU when there is one)."""
    from synth import make_problem
    from synth.generate import _default_device
    dev = _default_device()
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nact = int(rng.integers(4, 9))
        c, v, n = int(rng.integers(4, 43)), int(rng.integers(20, 351)), int(rng.integers(1, 5))
        nel = nact if nact % 2 == 0 else nact - 1
        out.append(make_problem(nclosed=c, nact=nact, nvirt=v, naux=3 * (c + nact + v),
                                nstate=n, seed=seed + k, nelact=nel, fast=True,
                                df_device=dev if dev != "cpu" else None))
    return out


def run_serve(nreq=256, rate=20.0, slots=4, seed=7, max_pending=16):
    """Submit nreq requests at Poisson arrival times with at most max_pending outstanding (a
    client blocks while the server holds that many; each queued request keeps a copy of its
    inputs in host memory), collect them in submission order on a second thread; latencies
    measured by the server (submit -> results ready)."""
    import queue
    import threading
    import paper_1606_01273_gb300 as cp
    pool = serve_problems()
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, nreq)
    picks = rng.integers(0, len(pool), nreq)
    srv = cp.Server(slots=slots)
    sem = threading.Semaphore(max_pending)
    tq = queue.Queue()
    outs, errors = [], []

    def collect():
        for _ in range(nreq):
            k, t = tq.get()
            try:
                outs.append(srv.wait(t))
            except cp.CASPT2Error as exc:
                p = pool[picks[k]]
                errors.append(f"{exc} at c{p.nclosed} a{p.nact} v{p.nvirt} n{p.nstate}")
            sem.release()

    th = threading.Thread(target=collect)
    th.start()
    t0 = time.perf_counter()
    tnext = t0
    for k in range(nreq):
        tnext += gaps[k]
        dt = tnext - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        sem.acquire()
        tk = srv.submit(pool[picks[k]], densities=(k % 2 == 0), xms=1, scheme=0, shift=0.2)
        tq.put((k, tk))
    th.join()
    span = time.perf_counter() - t0
    srv.close()
    lat = np.array([o["latency_ms"] for o in outs]) if outs else np.array([np.nan])
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "solves_per_s": len(outs) / span, "requests": nreq, "slots": slots,
            "max_outstanding": max_pending, "errors": len(errors),
            "first_error": errors[0] if errors else None, "workload": SERVE_DESC}


def oracle_rate_and_parity(p, want_parity=True):
    """(cpu_baseline dict, parity dict) for the workload: whole oracle solves when they take
    seconds, else the class-H sample scaled to a solve; parity against whole oracle solves
    or against the stored oracle results (tests/golden) when the inputs match."""
    from synth.fingerprint import input_fingerprint
    g = golden(WORKLOAD)
    if g is None or not g.get("oracle_seconds") or sum(g["oracle_seconds"].values()) < 120:
        ts, ref = time_oracle(p)
        base = {"value": len(ts) / sum(ts), "unit": "solves/s", "cores": cpu_cores(),
                "kind": "oracle",
                "sample": (f"{len(ts)} whole amplitude + lambda solve(s) of the workload "
                           "(setup, classes A-H, H^eff, lambda), numpy FP64")}
        return base, {"reference": "oracle solved in this run", "Ems": ref[1].tolist()}
    dt, frac = classh_sample(p)
    base = {"value": frac / dt, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": ("the oracle's class-H moment sums over 2 of the %d closed orbitals "
                       "(%.2f%% of the solve's algorithmic flops), %.1f s, scaled to a solve "
                       "by that fraction; the full oracle solve recorded with the stored "
                       "results took %.0f s on %d cores" % (
                           p.nclosed, 100.0 * frac, dt, sum(g["oracle_seconds"].values()),
                           g.get("host_cores", 0)))}
    par = {"reference": "stored oracle results (tests/golden/%s.json)" % WORKLOAD}
    if want_parity:
        fp = input_fingerprint(p)
        par["inputs_match"] = fp == g["fingerprint"]
        par["Ems"] = g["Ems"]
        par["golden"] = g
    return base, par


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    big = golden(WORKLOAD) is not None and sum(golden(WORKLOAD)["oracle_seconds"].values()) >= 120
    p = make_inputs(kmax=2 if big else 4)
    if big:
        step = lambda: classh_sample(p)
    else:
        step = lambda: (oracle_solve(p), None)
    for _ in range(args.warmup):
        step()
    ts, fr = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = step()
        ts.append(time.perf_counter() - t0)
        if big:
            ts[-1], fr_k = r
            fr.append(fr_k)
    total = sum(ts)
    value = (sum(fr) / total) if big else args.steps / total
    sample = ("class-H moment sums over 2 of the %d closed orbitals per step, each scaled to "
              "a solve by its share of the solve's algorithmic flops" % p.nclosed) if big else \
             ("%d whole amplitude + lambda solves of the workload" % args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "classes": "ABCDEFGH", "form": "oracle (numpy FP64)"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import paper_1606_01273_gb300 as cp
    from paper_1606_01273_gb300.shard import job_rate, max_over_ranks, sum_over_ranks

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    cp.lib()
    dens = BENCH[WORKLOAD]["densities"]

    p = make_inputs()
    host = cp.problem_inputs(p)
    h2d = sum(x.nbytes for x in host if x is not None)
    n = p.nstate
    # energies, per-class pieces and lambda (plus d1 and d2 when the step has densities;
    # GDF stays in HBM for the gradient contraction with the derivative integrals)
    d2h = 8 * (4 * n * n + 2 * n + 1 + 8 * (n * n + n)) + (2 * 8 * p.nmo * p.nmo if dens else 0)
    dev_in = [torch.from_numpy(x).to(dev) for x in host]   # f, B, rdm1-4
    popt = dict(OPTS, precision=cp.BF16X if args.precision == "bf16x" else cp.FP64,
                slices=args.slices)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def time_device(opts, steps, warmup):
        """W warm-up + K timed steps with inputs resident in HBM."""
        ctx = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **opts)
        ctx.set_inputs(*dev_in)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                ctx.solve(stream.cuda_stream)
                if dens:
                    ctx.compute_densities(stream=stream.cuda_stream)
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        rec = {"kern_ms": [], "tri": [], "gemm": [], "panel": [], "dens_ms": [], "launches": 0,
               "status": []}
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(dev.index) as clk:
            for k in range(steps):
                with torch.cuda.stream(stream):
                    flush.fill_(float(k))                # L2 flush outside the timed events
                    ev[k][0].record(stream)
                    st = ctx.solve(stream.cuda_stream)
                    if dens:
                        ctx.compute_densities(stream=stream.cuda_stream)
                    ev[k][1].record(stream)
                r = ctx.result(st)
                rec["status"].append(st)
                rec["dens_ms"].append(r.timings_ms[8])
                rec["kern_ms"].append(r.timings_ms[4])
                rec["tri"].append((r.timings_ms[5], r.timings_ms[6], r.timings_ms[7],
                                   r.timings_ms[9]))
                rec["gemm"].append(tuple(r.timings_ms[10:13]) if len(r.timings_ms) >= 13
                                   else (0.0, 0.0, 0.0))
                rec["panel"].append(tuple(r.timings_ms[13:16]) if len(r.timings_ms) >= 16
                                    else (0.0, 0.0, 0.0))
                rec["launches"] += r.launches
            torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        total = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        total = max_over_ranks(total, dev)
        rec.update(total_s=total, clk=clk.summary(), last=ctx.result(rec["status"][-1]),
                   warnings=ctx.status()["warnings"], min_den=ctx.status()["min_denominator"])
        ctx.close()
        return rec

    main = time_device(popt, args.steps, args.warmup)
    total_s, last = main["total_s"], main["last"]
    kern_ms, tri, dens_ms, launches, clk = (main["kern_ms"], main["tri"], main["dens_ms"],
                                            main["launches"], main["clk"])
    gemm = main["gemm"]
    panel = main["panel"]
    value = job_rate(sum_over_ranks(args.steps, dev), total_s)
    # the plain FP64 form and the end-to-end run take fewer steps than the headline when the
    # workload is large (each still after 3 warm-up steps)
    sec_steps = args.steps if not args.quick_compare else min(args.steps, 3)
    other = None
    if args.precision == "bf16x" and not args.no_compare:
        other = time_device(dict(OPTS, precision=cp.FP64), sec_steps, 3)

    # end to end through the C ABI with host buffers (pinned), H2D + D2H inside the timing
    del dev_in
    torch.cuda.empty_cache()
    pinned = [torch.from_numpy(x).pin_memory() for x in host]
    ctx_h = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate, **popt)

    def e2e_step():
        ctx_h.set_inputs(*pinned)
        st = ctx_h.solve()
        if dens:
            ctx_h.compute_densities()
        ctx_h.result(st)
        if dens:
            ctx_h.get_densities(with_gdf=False)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(sec_steps):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = job_rate(sum_over_ranks(sec_steps, dev), e2e_s)
    ctx_h.close()
    del pinned

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    kavg = statistics.mean(kern_ms)
    cv = p.nclosed * p.nvirt
    if args.precision == "bf16x":
        # algorithmic work of the class-H pair integrals, 2 (c v)^2 X flops, against the BF16
        # tensor peak (the 28 BF16 slice products of the exact split are reported beside it)
        flops = 2.0 * cv * cv * p.naux
        npair = args.slices * (args.slices + 1) // 2
        achieved = flops / (kavg * 1e-3) / 1e12
        peak, peak_kind = measured_peak("bf16_tflops", 1900.0)
        roof_h = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                  "frac": achieved / peak, "kernel": "k_oz_gemm", "kernel_ms": kavg,
                  "flops_per_launch": flops,
                  "tensor_pipe_tflops": npair * flops / (kavg * 1e-3) / 1e12,
                  "tensor_pipe_frac": npair * flops / (kavg * 1e-3) / 1e12 / peak,
                  "peak_kind": "bf16 burst, " + peak_kind}
    else:
        flops = classh_flops(p.nclosed, p.nvirt, p.naux)
        achieved = flops / (kavg * 1e-3) / 1e12
        roof_h = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                  "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                  "kernel": "k_classH", "kernel_ms": kavg,
                  "flops_per_launch": flops, "peak_kind": "nominal FP64"}
    tri_ms = sum(t[0] for t in tri)
    tri_fl = sum(t[1] for t in tri)
    tri_n = sum(t[2] for t in tri)
    tri_alg_bytes = sum(t[3] for t in tri) / max(tri_n, 1)
    tri_avg_ms = tri_ms / max(tri_n, 1)
    tri_achieved = tri_fl / max(tri_ms * 1e-3, 1e-12) / 1e12
    g_ms = sum(t[0] for t in gemm)
    g_fl = sum(t[1] for t in gemm)
    g_n = sum(t[2] for t in gemm)
    g_achieved = g_fl / max(g_ms * 1e-3, 1e-12) / 1e12
    p_ms = sum(t[0] for t in panel)
    p_by = sum(t[1] for t in panel)
    p_n = sum(t[2] for t in panel)
    p_gbs = p_by / max(p_ms * 1e-3, 1e-12) / 1e9
    hbm_peak, hbm_kind = measured_peak("hbm_gbs", 6800.0)
    sflops = solve_flops(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64 (bf16 slices on tensor cores)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "step": BENCH[WORKLOAD]["step"],
                   "classes": cp.supported_classes(),
                   "form": ("split-BF16 tensor-core products, %d slices (FP64-accurate), "
                            "FP64 eigensolvers and reductions" % args.slices
                            if args.precision == "bf16x" else "plain FP64"),
                   "parallelism": f"{ws} independent solve(s)",
                   "l2": "256 MB write between steps; B (%d MB) larger than L2" % (
                       p.B.nbytes // 2 ** 20)},
        "tflops_algorithmic": sflops / (total_s / args.steps) / 1e12,
        "solve_flops": sflops,
        # dominant kernel by device time (profiles/launches_c70a10v600x2000n5_*): the panel
        # kernel of the blocked Householder reduction, event-timed launch by launch inside
        # the solve; its algorithmic bytes are the trailing matrix its matrix-vector
        # products read, 8 n1^2 per column (64 columns per launch)
        "roofline": {"bound": "hbm", "achieved": p_gbs, "peak": hbm_peak, "unit": "GB/s",
                     "frac": p_gbs / hbm_peak, "traffic": None,
                     "kernel": "k_latrd", "kernel_ms": p_ms / max(p_n, 1),
                     "launches_per_step": p_n / max(len(panel), 1),
                     "alg_bytes_per_launch": p_by / max(p_n, 1),
                     "peak_kind": "HBM copy, " + hbm_kind},
        # the FP64 GEMM of the eigensolvers (blocked-reduction trailing updates, Z^T Z, the
        # small sectors' transforms), 2 M N K flops per launch, event-timed per launch
        "roofline_dgemm": {"bound": "alu", "achieved": g_achieved, "peak": FP64_PEAK_TFLOPS,
                           "unit": "TFLOP/s", "frac": g_achieved / FP64_PEAK_TFLOPS,
                           "kernel": "k_dgemm", "kernel_ms": g_ms / max(g_n, 1),
                           "launches_per_step": g_n / max(len(gemm), 1),
                           "flops_per_launch": g_fl / max(g_n, 1),
                           "peak_kind": "nominal FP64 (no measured FP64 peak in MEASURED_PEAKS)"},
        # the Householder tridiagonalisation (panels and their GEMM updates), 4/3 m^3 flops
        "roofline_tridiag": {"bound": "alu", "achieved": tri_achieved,
                             "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": tri_achieved / FP64_PEAK_TFLOPS,
                             "kernel": "k_latrd + k_dgemm / k_tridiag_smem",
                             "kernel_ms": tri_avg_ms,
                             "launches_per_step": tri_n / max(len(tri), 1),
                             "flops_per_launch": tri_fl / max(tri_n, 1),
                             "alg_bytes_per_launch": tri_alg_bytes,
                             "peak_kind": "nominal FP64"},
        "roofline_classH": roof_h,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": sec_steps},
        "gpu_launches": launches,
        "clocks": clk,
        "status": {"last": main["status"][-1], "warnings": main["warnings"],
                   "min_denominator_Eh": main["min_den"]},
        "fp64_form": None if other is None else {
            "value": ws * sec_steps / other["total_s"], "unit": "solves/s", "steps": sec_steps,
            "ms_per_step": 1e3 * other["total_s"] / sec_steps,
            "speedup_of_value": (ws * args.steps / total_s) / (ws * sec_steps / other["total_s"]),
            "max_abs_dE_vs_value_Eh": float(np.abs(other["last"].Ems - last.Ems).max()),
            "clocks": other["clk"]},
        "stage_ms_last": dict(zip(["setup", "classH", "classesAG", "heff_lambda", "classH_kernel",
                                   "tridiag_kernel_total"], last.timings_ms[:6]),
                              densities=statistics.mean(dens_ms) if dens else None),
    }
    if ws == 1 and args.precision == "bf16x" and not args.no_compare:
        # the error of fewer slices beside the FP64-accurate result: 1 slice is a single
        # BF16 pass of every split product (8-bit operands, FP32 accumulation)
        sp = {}
        for S in (1, 2, 3):
            ctx_s = cp.Context(p.nclosed, p.nact, p.nvirt, p.naux, p.nstate,
                               **dict(OPTS, precision=cp.BF16X, slices=S))
            host_s = cp.problem_inputs(p)
            ctx_s.set_inputs(*host_s)
            rs = ctx_s.result(ctx_s.solve())
            ctx_s.close()
            sp["%d_slice" % S] = {"max_abs_dE_vs_7_slices_Eh": float(np.abs(rs.Ems - last.Ems).max()),
                                  "max_rel_dE": float(np.abs(rs.Ems - last.Ems).max()
                                                      / np.abs(last.Ems).max())}
        line["fewer_slices"] = sp
    if ws == 1 and not args.no_cpu_baseline:
        base, par = oracle_rate_and_parity(p)
        line["cpu_baseline"] = base
        ref = np.asarray(par["Ems"])
        err = float(np.abs(last.Ems - ref).max())
        par_out = {"reference": par["reference"], "max_abs_dE_Eh": err,
                   "max_rel_dE": err / float(np.abs(ref).max()), "tol_Eh": 1e-8}
        if "golden" in par:
            par_out["inputs_match"] = par["inputs_match"]
            par_out["conditioning_bound_Eh"] = conditioning_bound(par["golden"], OPTS["shift"])
        if other is not None:
            par_out["fp64_form_max_abs_dE_Eh"] = float(np.abs(other["last"].Ems - ref).max())
        line["parity"] = par_out
    if ws == 1 and not args.no_serve:
        # the serving stream last, with the workload's host arrays released
        del p, host
        import gc
        gc.collect()
        torch.cuda.empty_cache()
        line["serve"] = run_serve()
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# class masks (bit k = class "ABCDEFGH"[k]) for kernel captures: class A alone makes the
# first tridiagonalisation the 1536 x 1536 class-A overlap matrix; class H alone makes the
# first split GEMM the class-H pair-integral product K = Bcv^T Bcv (4000 x 4000 x 700)
PROFILE_CASES = {"classA": 1 << 0, "classH": 1 << 7, "sector2048": 1 << 0,
                 "classG": 1 << 6}


def run_profile_case(args):
    """Small commands for kernel captures (each a few GB on the device at most):
    classA / classH / classG: one solve of the selected workload restricted to that class;
    sector2048: class A of a c2 a8 v3 X40 n4 problem, whose 2048-wide overlap and Fock
    sectors take the blocked tridiagonalisation and the compact-WY back-transformation."""
    import paper_1606_01273_gb300 as cp
    prec = cp.BF16X if args.precision == "bf16x" else cp.FP64
    if args.profile_case == "sector2048":
        from synth import make_problem
        p = make_problem(nclosed=2, nact=8, nvirt=3, naux=40, nstate=4, seed=17, fast=True)
        r = cp.solve_problem(p, class_mask=1 << 0, precision=prec, slices=args.slices, xms=1,
                             scheme=0, shift=1.0)
    else:
        p = make_inputs()
        r = cp.solve_problem(p, class_mask=PROFILE_CASES[args.profile_case], precision=prec,
                             slices=args.slices, **OPTS)
    print("profile case", args.profile_case, "E_MS", list(np.round(r.Ems, 10)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--precision", choices=["fp64", "bf16x"], default="bf16x")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--slices", type=int, default=7)
    ap.add_argument("--workload", choices=sorted(BENCH), default=DEFAULT_WORKLOAD)
    ap.add_argument("--quick-compare", action="store_true", default=None,
                    help="the FP64-form and end-to-end arms take min(steps, 3) steps "
                         "(default on for the copper-corrole workload)")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES),
                    help="one solve of the benchmark workload restricted to one class (a "
                         "small command for kernel captures); prints no JSON line")
    args = ap.parse_args()
    global WORKLOAD, OPTS, WORKLOAD_DESC
    WORKLOAD = args.workload
    OPTS = BENCH[WORKLOAD]["opts"]
    WORKLOAD_DESC = BENCH[WORKLOAD]["desc"]
    if args.quick_compare is None:
        args.quick_compare = WORKLOAD == "c70a10v600x2000n5"
    if args.profile_case:
        return run_profile_case(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

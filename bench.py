#!/usr/bin/env python
"""Throughput of the GE node-vector distance on GB300.

Workload (one "step", the default line): the erased configuration-model graph
with n = 10,000,000 nodes and a power-law degree sequence (exponent 2.3 on
[2, 10,000], largest component, lognormal(0,1) FP32 weights) and 128 vector pairs
whose x and y have Uniform[0,1) values on 0.1% of the nodes, normalised to sum 1.
All 128 distances d^2 = delta^T L^+ delta (Section 3.1 GE equation via the
Laplacian solve of Section 3.2) are computed by FP32 block-PCG (32 right-hand
sides per SpMM) inside an FP64 iterative-refinement loop to d^2 relative change
1e-8.  Inputs are seeded and synthetic (no dataset).

Metric: GE distances per second (whole job).  Beside it: the live roofline of the
FP32 multi-column SpMM (algorithmic bytes / CUDA-event time of its launches in the
timed region, against the measured HBM copy bandwidth), the end-to-end rate
through the C ABI with host buffers, the oracle (plain FP64 CPU CG) timed on this
machine's cores, and the other workloads' headline numbers (the n = 10^6
Erdos-Renyi graph solved one right-hand side at a time in FP64, the multiple of
batched mixed precision over it, and the power-law graph after exact elimination
of its degree-1/2 nodes).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload powerlaw|er_large|batched|grad|resistance|resistance_matrix]

With N > 1 (torchrun, one rank per GPU) every rank solves its own 128 pairs on its
own copy of the graph (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GE distances/s on 1 GB300 at d² rel.err≤1e-6; SpMV HBM GB/s vs peak"
UNIT = "distances/s"
PL_PAIRS = 128         # power-law workload: pairs per step (per rank)
PL_RTOL_IN = 5e-5      # its inner FP32 solve tolerance
PL_D2_RTOL = 1e-8      # its refinement stop (relative change of d^2)
PL_ORACLE_PAIRS = 2    # pairs the oracle solves for the CPU baseline and the error check
PAIRS_PER_STEP = 8
RTOL = 1e-10
CHECK_EVERY = 2   # PCG iterations between the host's convergence polls (polled one batch behind)
SPMV_SAMPLE = 4   # the live SpMV timer brackets one launch in 4 (events break launch overlap)
MIXED_RTOL_IN = 1e-4   # inner FP32 solve tolerance of the mixed-precision comparison
MIXED_D2_RTOL = 1e-8   # its refinement stop (relative change of d^2)
D2_STOP_RTOL = 1e-6    # the d^2 accuracy the metric states, for the d^2-stop comparison


def workload_config(g, n0):
    return {
        "workload": "er_large: Erdos-Renyi G(n=1e6, m=5e6) largest component, FP64 weights "
                    "U[0.5,2), 8 pairs x,y U[0,1) on 1% of nodes normalised, single-RHS FP64 "
                    "Jacobi-PCG to relative residual 1e-10",
        "n": int(g.n), "nnz": int(g.nnz), "n_generated": int(n0), "pairs_per_step": PAIRS_PER_STEP,
        "rtol": RTOL, "solver": "FP64 PCG, one right-hand side at a time", "check_every": CHECK_EVERY,
        "l2": "L2 flushed (256 MB write) between timed steps; working set 0.3 GB > 129 MB L2",
    }


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_pair_range(rank):
    """First pair index and count of a rank's share (ranks take disjoint pairs: weak scaling)."""
    return rank * PAIRS_PER_STEP, PAIRS_PER_STEP


def job_time(local, dist=None, device=None):
    """The job's time: the maximum of the ranks' times (one all-reduce; none on one rank)."""
    if dist is None:
        return float(local)
    import torch
    t = torch.tensor([float(local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, steps, total_ms):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world * steps / (total_ms / 1e3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


SPMV_SOURCES = ("paper_2310_11222_gb300/csrc/kernels.cuh", "paper_2310_11222_gb300/csrc/common.h",
                "paper_2310_11222_gb300/csrc/solver.cuh", "paper_2310_11222_gb300/csrc/graph.cu")
SPMM_STREAM_SOURCES = SPMV_SOURCES + ("paper_2310_11222_gb300/csrc/tma.cuh", "paper_2310_11222_gb300/csrc/stream.cuh")


def kernel_source_hash(sources=SPMV_SOURCES):
    """Hash of the sources that decide a kernel's code and its work layout."""
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(name="spmv_er_large_traffic.txt", sources=SPMV_SOURCES):
    """DRAM bytes per launch from a committed ncu summary under profiles/, if it was
    taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    d = {}
    with open(p) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    if d.get("kernel_source_hash") != kernel_source_hash(sources):
        return None
    try:
        return float(d["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        idx = str(local_rank)
        if vis:
            parts = [p.strip() for p in vis.split(",") if p.strip()]
            if local_rank < len(parts):
                idx = parts[local_rank]
        self.idx = idx
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.idx], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(g, X, Y, budget_s=12.0, max_solves=200):
    """The oracle (plain FP64 CPU Jacobi-PCG, oracle/pcg.c) on this host's cores over a
    bounded sample of the same pairs (the given pairs in turn, repeated until about
    budget_s of CPU work, every pair at least once): returns (distances/s, threads,
    solves, seconds, d2 of the first pass over the pairs)."""
    import numpy as np
    from oracle import cg as ocg
    ocg.build()
    threads = ocg.default_threads()
    k = X.shape[0]
    t0 = time.perf_counter()
    d2s = []
    solves = 0
    while solves < max_solves:
        j = solves % k
        d2, it, rr = ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X[j:j + 1], Y[j:j + 1],
                                  rtol=RTOL, threads=threads)
        if solves < k:
            d2s.append(float(d2[0]))
        solves += 1
        if time.perf_counter() - t0 >= budget_s and solves >= min(k, max_solves):
            break
    dt = time.perf_counter() - t0
    return solves / dt, threads, solves, dt, d2s


def run_other_workload(args, nvd, synth, torch, np, local):
    """Measurement of the other workloads of the method (not the default bench line):
    the 64-graph batched workload (one persistent graph-captured launch), the
    differentiation workload (forward + adjoint backward), effective resistances on
    node-id pairs and the resistance matrix of a node subset.  Same JSON fields as
    the default line."""
    from oracle import cg as ocg
    dev = torch.device("cuda", local)
    name = args.workload
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prof = True
    tuning = None
    if name == "batched":
        wl = synth.workload_batched()
        graphs = wl.graphs
        X, Y = wl.pairs(0, 32)
        Gs = [nvd.Graph.from_csr(gi) for gi in graphs]
        xs = [torch.from_numpy(x).to(dev) for x in X]
        ys = [torch.from_numpy(y).to(dev) for y in Y]
        xhs = [torch.from_numpy(x).pin_memory() for x in X]
        yhs = [torch.from_numpy(y).pin_memory() for y in Y]
        k = 32 * len(graphs)
        # the workload as stated: one persistent, graph-captured launch; the library's
        # default host-driven form is timed beside it (batched_host_loop)
        kw = dict(mode=nvd.MODE_FP32, rtol=1e-6, persistent=True)
        prof = False   # one persistent launch per step: no separate SpMM launches to time

        def step():
            return nvd.ge_distance_batched(Gs, xs, ys, **kw)

        def step_e2e():
            for a, b in zip(xs, xhs):
                a.copy_(b, non_blocking=True)
            for a, b in zip(ys, yhs):
                a.copy_(b, non_blocking=True)
            return nvd.ge_distance_batched(Gs, xs, ys, **kw)
        h2d, d2h = sum(2 * x.nbytes for x in X), 8 * k
        cfg = {"workload": "batched: 64 graphs, n log-uniform in [1e3, 2e5], 32 BA (m in 2..6) + 32 WS "
                           "(k=10, p=0.1), unit weights, 32 pairs each (16 e_i - e_j, 16 diffuse); FP32 "
                           "block-PCG with FP64 reductions to rtol 1e-6, the 64 graphs as one block-diagonal "
                           "Laplacian in one persistent graph-captured launch",
               "graphs": len(graphs), "n_total": int(sum(gi.n for gi in graphs)),
               "nnz_total": int(sum(int(gi.rowptr[-1]) for gi in graphs)), "pairs_per_step": k}
        unit = UNIT
        dtype = "f32+f64"

        def oracle_sample():
            t0 = time.perf_counter()
            done = 0
            for gi, x, y in zip(graphs, X, Y):
                ocg.ge_d2_cg(gi.n, gi.rowptr, gi.colidx, gi.w.astype(np.float64), x, y, rtol=1e-6)
                done += x.shape[0]
                if time.perf_counter() - t0 > 10:
                    break
            return done / (time.perf_counter() - t0), f"{done} pairs of the first graphs, FP64 oracle CG at rtol 1e-6"
    elif name == "grad":
        wl = synth.workload_grad()
        g = wl.graph
        k = 64
        X, Y = wl.pairs(0, k)
        G = nvd.Graph.from_csr(g)
        if not args.no_tune:
            tuning = G.tune(mode=nvd.MODE_FP64, k=k)
        w = torch.from_numpy(g.w).to(dev).requires_grad_(True)
        xt = torch.from_numpy(X).to(dev).requires_grad_(True)
        yt = torch.from_numpy(Y).to(dev)
        xh, yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()

        def step():
            w.grad = None
            xt.grad = None
            d2 = nvd.ge_distance_autograd(G, xt, yt, w, rtol=RTOL)
            d2.sum().backward()
            return d2

        def step_e2e():
            with torch.no_grad():
                xt.copy_(xh, non_blocking=True)
                yt.copy_(yh, non_blocking=True)
            d2 = step()
            return d2.detach().cpu()
        h2d, d2h = 2 * X.nbytes, 8 * k
        cfg = {"workload": "grad: BA n=1e6 m=5, lognormal(0,0.5) FP32 weights with requires_grad, 64 pairs "
                           "U[0,1) on 10% of nodes; forward FP64 PCG to rtol 1e-10 plus the adjoint backward "
                           "(grad_w, grad_x)", "n": g.n, "nnz": int(g.rowptr[-1]), "pairs_per_step": k,
               "tuning": tuning}
        unit = "pairs/s (forward + backward)"
        dtype = "f64"

        def oracle_sample():
            t0 = time.perf_counter()
            ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), X[:1], Y[:1], rtol=RTOL, return_z=True)
            return 1.0 / (time.perf_counter() - t0), "1 pair forward (z), FP64 oracle CG at rtol 1e-10"
    elif name == "resistance":
        wl = synth.workload_er_large()
        g = wl.graph
        k = 256
        rng = np.random.default_rng(2024)
        U = rng.integers(0, g.n, k).astype(np.int32)
        V = ((U + 1 + rng.integers(0, g.n - 1, k)) % g.n).astype(np.int32)
        G = nvd.Graph.from_csr(g)
        if not args.no_tune:
            tuning = G.tune(mode=nvd.MODE_FP64, k=k)

        def step():
            return nvd.effective_resistance(G, U, V, rtol=RTOL)
        step_e2e = step                      # ids and results are host arrays in the call itself
        h2d, d2h = 2 * 4 * k, 8 * k
        cfg = {"workload": "resistance: effective resistance R(u,v) of 256 seeded node pairs on the ER graph "
                           "(n=1e6 generated, largest component, mean degree 10, U[0.5,2] FP64 weights); "
                           "right-hand sides e_u - e_v built on the device from the ids, FP64 block-PCG to "
                           "rtol 1e-10; host ids in, host results out inside the timed call",
               "n": g.n, "nnz": int(g.rowptr[-1]), "pairs_per_step": k, "tuning": tuning}
        unit = "resistances/s"
        dtype = "f64"

        def oracle_sample():
            x = np.zeros((1, g.n))
            y = np.zeros((1, g.n))
            x[0, U[0]] = 1.0
            y[0, V[0]] = 1.0
            t0 = time.perf_counter()
            ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), x, y, rtol=RTOL)
            return 1.0 / (time.perf_counter() - t0), "1 node pair (indicator vectors), FP64 oracle CG at rtol 1e-10"
    elif name == "resistance_matrix":
        wl = synth.workload_er_large()
        g = wl.graph
        s_n = 256
        nodes = np.random.default_rng(2025).choice(g.n, s_n, replace=False).astype(np.int32)
        k = s_n * (s_n - 1) // 2                 # distinct node pairs of the matrix
        G = nvd.Graph.from_csr(g)
        if not args.no_tune:
            tuning = G.tune(mode=nvd.MODE_FP64, k=s_n - 1)

        def step():
            return nvd.resistance_matrix(G, nodes, rtol=RTOL)
        step_e2e = step                      # ids and the matrix are host arrays in the call itself
        h2d, d2h = 4 * s_n, 8 * s_n * s_n
        cfg = {"workload": "resistance_matrix: effective-resistance matrix of 256 seeded nodes of the ER graph "
                           "(n=1e6 generated, largest component, mean degree 10, U[0.5,2] FP64 weights): 255 "
                           "FP64 block-PCG solves L z_d = e_d - e_r to rtol 1e-10, then R(a,b) from the z "
                           "entries at the subset; value counts the 32,640 distinct pairs per matrix",
               "n": g.n, "nnz": int(g.rowptr[-1]), "subset": s_n, "solves_per_step": s_n - 1,
               "pairs_per_step": k, "tuning": tuning}
        unit = "resistances/s"
        dtype = "f64"

        def oracle_sample():
            x = np.zeros((1, g.n))
            y = np.zeros((1, g.n))
            x[0, nodes[1]] = 1.0
            y[0, nodes[0]] = 1.0
            t0 = time.perf_counter()
            ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, g.w.astype(np.float64), x, y, rtol=RTOL)
            return 1.0 / (time.perf_counter() - t0), ("1 node pair per oracle CG solve at rtol 1e-10 (the oracle "
                                                       "has no subset shortcut)")
    else:
        raise SystemExit(f"unknown workload {name}")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if prof:
        nvd.profile_enable(True)
        nvd.profile_read(0)
    launches0 = nvd.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for s_ in range(args.steps):
        flush.zero_()
        ev[s_][0].record()
        step()
        ev[s_][1].record()
    torch.cuda.synchronize()
    launches = nvd.kernel_launches() - launches0
    n_spmv, spmv_ms, spmv_bytes = nvd.profile_read(0) if prof else (0, 0.0, 0.0)
    nvd.profile_enable(False)
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    te0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    torch.cuda.synchronize()
    te = time.perf_counter() - te0
    peaks, peak_src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = (spmv_bytes / n_spmv) / (spmv_ms / n_spmv / 1e3) / 1e9 if n_spmv else None
    value = k * args.steps / (total_ms / 1e3)
    step_roof = None
    if name == "batched":
        # the whole step against the copy bandwidth: per graph, the iterations its
        # slowest column ran times one PCG iteration's bytes (SpMM: CSR entries, row
        # pointers, degrees, p read, q written; residual pass: r, q read, r written,
        # D^-1; direction pass: x, r, p read, x, p written, D^-1), FP32 values, 32 columns
        _, st = nvd.ge_distance_batched(Gs, xs, ys, return_stats=True, **kw)
        kt, sv = 32, 4
        tot_bytes, off = 0.0, 0
        for gi, x in zip(graphs, X):
            its = max(s_["iters"] for s_ in st[off:off + x.shape[0]])
            off += x.shape[0]
            n_, nnz_ = gi.n, int(gi.rowptr[-1])
            per_it = (nnz_ * (4 + sv) + 8 * (n_ + 1) + n_ * sv + 2 * n_ * kt * sv) + 8 * n_ * kt * sv + 2 * n_ * sv
            tot_bytes += its * per_it
        ach = tot_bytes / (total_ms / args.steps / 1e3) / 1e9
        step_roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                     "traffic": None,
                     "kernel": "k_persistent<float,float,float,32,float> (the whole batch: SpMM and vector passes "
                               "of every graph's PCG iterations in one launch per step; duration = the step's "
                               "event time)",
                     "launches": args.steps, "avg_launch_us": 1e3 * total_ms / args.steps,
                     "algorithmic_bytes_per_launch": tot_bytes,
                     "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy) of MEASURED_PEAKS.json"}
        # the library's default form (host-driven launches over all graphs), same
        # pairs, same process: its rate and its SpMM launches' roofline
        kh = dict(kw, persistent=False)
        for _ in range(args.warmup):
            nvd.ge_distance_batched(Gs, xs, ys, **kh)
        torch.cuda.synchronize()
        nvd.profile_enable(True)
        nvd.profile_read(0)
        evh = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a_, b_ in evh:
            flush.zero_()
            a_.record()
            nvd.ge_distance_batched(Gs, xs, ys, **kh)
            b_.record()
        torch.cuda.synchronize()
        nh, hms, hbytes = nvd.profile_read(0)
        nvd.profile_enable(False)
        tot_h = sum(a_.elapsed_time(b_) for a_, b_ in evh)
        host_line = {"distances_per_s": k * args.steps / (tot_h / 1e3), "ms_per_step": tot_h / args.steps,
                     "vs_persistent": total_ms / tot_h,
                     "spmm_roofline": {"frac": ((hbytes / nh) / (hms / nh / 1e3) / 1e9) / peak if nh else None,
                                       "avg_launch_us": 1e3 * hms / nh if nh else None, "launches": nh},
                     "what": "nvd_ge_distance_batched default: one launch per phase over all graphs, the host "
                             "polling convergence"}
    line = {
        "metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg,
        "e2e": {"value": k * args.steps / te, "unit": unit, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches), "clocks": clk,
        "roofline": step_roof if step_roof is not None else None if not n_spmv else {
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_spmm (every SpMV/SpMM launch of the step, algorithmic bytes)",
            "launches": n_spmv, "avg_launch_us": 1e3 * spmv_ms / n_spmv,
            "algorithmic_bytes_per_launch": spmv_bytes / n_spmv,
            "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy) of MEASURED_PEAKS.json"},
    }
    if step_roof is not None:
        line["batched_host_loop"] = host_line
    if not args.no_cpu_baseline:
        v, what = oracle_sample()
        line["cpu_baseline"] = {"value": v, "unit": unit, "cores": ocg.default_threads(), "kind": "oracle",
                                "sample": what}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, nvd, synth, torch, np, local):
    """The paper's synthetic experiments (Section 4.2) on this GPU: time of one GE
    evaluation (one pair, FP64 PCG to relative residual 1e-10, single right-hand side,
    graph tuned beforehand) against |V| at mean degree 8 (size) or against the mean
    degree at |V| = 10^4 (density), for ER, BA, WS and SBM graphs with the same number
    of edges.  Ten runs per point; runs longer than twice the mean are dropped (the
    paper's rule).  Prints one JSON line per point and one summary line with the
    fitted exponent of time against |V| (size sweep, |V| >= 10^4)."""
    dev = torch.device("cuda", local)
    if args.sweep == "size":
        points = [(n, 8.0) for n in (1000, 10000, 100000, 1000000)]
    else:
        points = [(10000, float(k)) for k in (1, 2, 4, 8, 16, 32, 64)]
    rows = []
    for model in ("er", "ba", "ws", "sbm"):
        for n, kdeg in points:
            if model in ("ba", "ws") and kdeg < 2:
                continue
            g = synth.sweep_graph(model, n, kdeg, seed=n + int(kdeg))
            X, Y = synth.sparse_uniform_pairs(g.n, 1, 0.10, 5000 + n)
            G = nvd.Graph.from_csr(g)
            G.tune(mode=nvd.MODE_FP64, k=1, single_rhs=True)
            xt, yt = torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)
            for _ in range(3):
                nvd.ge_distance(G, xt, yt, rtol=RTOL, single_rhs=True)
            torch.cuda.synchronize()
            times = []
            for _ in range(10):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                d2, st = nvd.ge_distance(G, xt, yt, rtol=RTOL, single_rhs=True, return_stats=True)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            mean = sum(times) / len(times)
            kept = [t for t in times if t <= 2 * mean]
            row = {"sweep": args.sweep, "model": model, "n": g.n, "mean_degree": kdeg,
                   "nnz": int(g.rowptr[-1]), "ms_mean": sum(kept) / len(kept),
                   "ms_median": statistics.median(times), "iters": st[0]["iters"],
                   "d2": float(d2[0])}
            rows.append(row)
            print(json.dumps(row), flush=True)
            del G
    if args.sweep == "size":
        fits = {}
        for model in ("er", "ba", "ws", "sbm"):
            pts = [(r["n"], r["ms_mean"]) for r in rows if r["model"] == model and r["n"] >= 10000]
            if len(pts) >= 2:
                lx = np.log([p[0] for p in pts])
                ly = np.log([p[1] for p in pts])
                fits[model] = float(np.polyfit(lx, ly, 1)[0])
        print(json.dumps({"sweep": "size", "exponent_time_vs_V": fits}), flush=True)
    return 0


def run_reference(args):
    """Reference arm: the oracle (plain FP64 CPU Jacobi-PCG, oracle/pcg.c) timed as it
    stands on the host cores, on the same workload as the default line; one step is a
    bounded sample of it: one pair solved to rtol 1e-10 (rank 0 only)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import numpy as np
    import synth
    from oracle import cg as ocg
    if args.workload == "er_large":
        wl = synth.workload_er_large()
        g = wl.graph
        per = PAIRS_PER_STEP
        cfg = workload_config(g, wl.meta["n_generated"])
    else:
        wl = synth.workload_powerlaw(scale=args.scale)
        g = wl.graph
        per = PL_PAIRS
        cfg = powerlaw_config(g, wl, args, None, None)
    X, Y = wl.pairs(0, per)
    w64 = g.w.astype(np.float64)
    ocg.build()
    threads = ocg.default_threads()
    for s in range(args.warmup):
        j = s % per
        ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, w64, X[j:j + 1], Y[j:j + 1], rtol=RTOL, threads=threads)
    t0 = time.perf_counter()
    for s in range(args.steps):
        j = (args.warmup + s) % per
        ocg.ge_d2_cg(g.n, g.rowptr, g.colidx, w64, X[j:j + 1], Y[j:j + 1], rtol=RTOL, threads=threads)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.steps} pairs of the workload, one per step, oracle FP64 CG "
                                   f"(oracle/pcg.c) at rtol 1e-10"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def powerlaw_config(g, wl, args, tuning, elim):
    return {
        "workload": "powerlaw: erased configuration model n=1e7, degree exponent 2.3 on [2, 1e4], largest "
                    "component, lognormal(0,1) FP32 weights, 128 pairs x,y U[0,1) on 0.1% of nodes normalised; "
                    f"FP32 block-PCG (32 right-hand sides per SpMM, rtol {PL_RTOL_IN}) inside FP64 iterative "
                    f"refinement to d^2 relative change {PL_D2_RTOL}"
                    + ("; degree-1/2 nodes eliminated exactly, PCG on the reduced graph" if args.eliminate else ""),
        "n": int(g.n), "nnz": int(g.rowptr[-1]), "n_generated": int(wl.meta["n_generated"]),
        "pairs_per_step": PL_PAIRS, "mode": "MIXED", "rtol_inner": PL_RTOL_IN, "d2_rtol": PL_D2_RTOL,
        "graph_storage": "degree-ordered inside the component (NVD_GRAPH_REORDER_DEGREE, set-up)",
        "scale": args.scale, "tuning": tuning, "elimination": elim,
        "l2": "L2 flushed (256 MB write) between timed steps; working set ~30 GB > 129 MB L2",
    }


def run_powerlaw(args, nvd, synth, torch, np, rank, world, local, dist):
    """The default line: the power-law precision workload, 128 pairs per step (per rank),
    FP32 block-PCG inside FP64 refinement (MIXED), inputs resident on the device."""
    dev = torch.device("cuda", local)
    wl = synth.workload_powerlaw(scale=args.scale)
    g = wl.graph
    X, Y = wl.pairs(rank * PL_PAIRS, PL_PAIRS)                 # each rank its own pairs
    # stored degree-ordered inside the component (NVD_GRAPH_REORDER_DEGREE): the hub
    # rows the SpMM gathers most are one contiguous run and light blocks hold rows of
    # similar length; results come back in the caller's node order
    G = nvd.Graph.from_csr(g, reorder=True)
    # work decomposition picked by the autotuner on this graph (set-up, not timed)
    if args.tuning:
        # a fixed setting (profiling runs repeat the bench's tuned decomposition)
        tuning = dict(json.loads(args.tuning))
        G.set_tuning(mode=nvd.MODE_MIXED, **tuning)
        tuning["source"] = "--tuning"
    else:
        tuning = None if args.no_tune else G.tune(mode=nvd.MODE_MIXED, k=PL_PAIRS)
    elim = G.eliminate() if args.eliminate else None
    xt = torch.from_numpy(X).to(dev)
    yt = torch.from_numpy(Y).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    kw = dict(mode=nvd.MODE_MIXED, rtol=PL_RTOL_IN, d2_rtol=PL_D2_RTOL, eliminate=args.eliminate)

    def step():
        return nvd.ge_distance(G, xt, yt, return_stats=True, **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    nvd.profile_enable(True)
    for cls in (0, 1, 2):
        nvd.profile_read(cls)
    launches0 = nvd.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall0 = time.perf_counter()
    last = None
    for k in range(args.steps):
        flush.zero_()                                   # evict L2 between steps (not timed)
        ev[k][0].record()
        last = step()
        ev[k][1].record()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = nvd.kernel_launches() - launches0
    n_spmm, spmm_ms, spmm_bytes = nvd.profile_read(0)
    n_res, res_ms, res_bytes = nvd.profile_read(2)
    nvd.profile_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = job_time(sum(step_ms), dist, dev)
    d2_last, stats = last

    # ---- end to end through the C ABI: pinned host x, y copied to the device inside
    #      the call (overlapped with the previous tile's solve), d^2 back to the host
    xh = torch.from_numpy(X).pin_memory()
    yh = torch.from_numpy(Y).pin_memory()

    def step_e2e():
        if args.eliminate:                # the elimination path takes device inputs
            xt.copy_(xh, non_blocking=True)
            yt.copy_(yh, non_blocking=True)
            return nvd.ge_distance(G, xt, yt, **kw).cpu()
        return nvd.ge_distance(G, xh, yh, **kw)

    step_e2e()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        d2_host = step_e2e()
    torch.cuda.synchronize()
    te = job_time(time.perf_counter() - te0, dist, dev)

    value = job_rate(PL_PAIRS, world, args.steps, total_ms)
    peaks, peak_src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = (spmm_bytes / n_spmm) / (spmm_ms / n_spmm / 1e3) / 1e9 if n_spmm else None
    gather = 0 if tuning is None else int(tuning.get("gather", 0))
    folded = bool(tuning and tuning.get("fold_direction"))
    kt = (tuning or {}).get("kt") or 32
    kbase = {0: "k_spmm", 1: "k_spmm_stream", 2: "k_spmm_tma"}[gather]
    # the committed DRAM count is of one full-size launch of this decomposition
    traffic = (ncu_traffic(f"spmm_powerlaw_kt{kt}_g{gather}_traffic.txt", SPMM_STREAM_SOURCES)
               if not folded and args.scale == 1.0 and not args.eliminate else None)
    kname = (f"{kbase}<float,float,float,{kt},{'EpiLapDir' if folded else 'EpiLap'}> (FP32 multi-column "
             f"Laplacian SpMM, {['register loads per slice', 'register loads over each warp stream', 'TMA gathers over each warp stream'][gather]}, fused p^T q)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": powerlaw_config(g, wl, args, tuning, elim),
        "e2e": {"value": job_rate(PL_PAIRS, world, args.steps, 1e3 * te), "unit": UNIT,
                "h2d_bytes_per_step": int(xh.numel() * 8 * 2), "d2h_bytes_per_step": PL_PAIRS * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": kname, "launches": n_spmm,
                     "avg_launch_us": 1e3 * spmm_ms / n_spmm if n_spmm else None,
                     "algorithmic_bytes_per_launch": spmm_bytes / n_spmm if n_spmm else None,
                     # the DRAM bytes the ncu summary counted per launch over the live launch
                     # time: the bandwidth the kernel sustains on its real (gather-heavy) traffic
                     "traffic_gbs": traffic / (spmm_ms / n_spmm / 1e3) / 1e9 if traffic and n_spmm else None,
                     "traffic_frac": traffic / (spmm_ms / n_spmm / 1e3) / 1e9 / peak if traffic and n_spmm else None,
                     "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy) of MEASURED_PEAKS.json"},
        "solver": {"inner_iters_per_pair": [s_["iters"] for s_ in stats],
                   "refine_steps": sorted({s_["refine_steps"] for s_ in stats}),
                   "status": sorted({s_["status"] for s_ in stats}), "wall_s_timed": t_wall,
                   "spmm_ms_per_step": spmm_ms / args.steps,
                   "residual_spmm": {"launches": n_res, "ms_per_step": res_ms / args.steps,
                                     "algorithmic_bytes_per_launch": res_bytes / n_res if n_res else None}},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Xo, Yo = X[:PL_ORACLE_PAIRS], Y[:PL_ORACLE_PAIRS]
        v, th, nsolves, dt, d2_or = cpu_baseline(g, Xo, Yo, budget_s=10.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                                "sample": f"{nsolves} solves over the step's first {len(d2_or)} pairs ({dt:.1f} s), "
                                          f"oracle FP64 Jacobi-PCG (oracle/pcg.c) at rtol 1e-10"}
        got = d2_last.cpu().numpy()[:len(d2_or)]
        line["max_rel_err_vs_oracle"] = float(np.max(np.abs(got - d2_or) / np.abs(d2_or)))
        line["max_rel_err_e2e_vs_oracle"] = float(np.max(np.abs(d2_host.numpy()[:len(d2_or)] - d2_or)
                                                         / np.abs(d2_or)))
    if rank == 0 and not args.no_extra:
        line["other_workloads"] = powerlaw_extras(args, nvd, synth, torch, np, dev, G, xt, yt, kw, d2_last)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def powerlaw_extras(args, nvd, synth, torch, np, dev, G, xt, yt, kw, d2_ref):
    """The other headline numbers, measured in the same process: the Erdos-Renyi
    workload solved one right-hand side at a time in FP64 (the plain method at scale)
    against batched mixed precision on the same graph and pairs (the stated
    multiple), and the power-law solve on the graph reduced by exact elimination of
    its degree-1/2 nodes."""
    out = {}

    def rate(Gh, x, y, k, reps, **kw2):
        nvd.ge_distance(Gh, x, y, **kw2)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            res = nvd.ge_distance(Gh, x, y, **kw2)
        b.record()
        torch.cuda.synchronize()
        return k * reps / (a.elapsed_time(b) / 1e3), res

    wl = synth.workload_er_large()
    ge = wl.graph
    Xe, Ye = wl.pairs(0, PAIRS_PER_STEP)
    Ge = nvd.Graph.from_csr(ge)
    xe, ye = torch.from_numpy(Xe).to(dev), torch.from_numpy(Ye).to(dev)
    t_single = None if args.no_tune else Ge.tune(mode=nvd.MODE_FP64, k=PAIRS_PER_STEP, single_rhs=True)
    r1, d1 = rate(Ge, xe, ye, PAIRS_PER_STEP, 5, rtol=RTOL, single_rhs=True, check_every=CHECK_EVERY)
    t_mixed = None if args.no_tune else Ge.tune(mode=nvd.MODE_MIXED, k=PAIRS_PER_STEP)
    rm, dm = rate(Ge, xe, ye, PAIRS_PER_STEP, 5, mode=nvd.MODE_MIXED, rtol=MIXED_RTOL_IN, d2_rtol=MIXED_D2_RTOL)
    d1, dm = d1.cpu().numpy(), dm.cpu().numpy()
    out["er_large"] = {
        "workload": "Erdos-Renyi G(n=1e6, m=5e6) largest component, FP64 weights U[0.5,2), 8 pairs on 1% of nodes",
        "fp64_single_rhs_distances_per_s": r1,
        "mixed_multi_rhs_distances_per_s": rm,
        "multiple_mixed_vs_single_rhs_fp64": rm / r1,
        "mixed": f"FP32 block-PCG to rtol {MIXED_RTOL_IN} inside FP64 refinement to d2_rtol {MIXED_D2_RTOL}",
        "max_rel_diff_mixed_vs_fp64": float(np.max(np.abs(dm - d1) / np.abs(d1))),
        "tuning_single": t_single, "tuning_mixed": t_mixed}
    del Ge
    if not args.eliminate:
        t0 = time.perf_counter()
        info = G.eliminate()
        t_elim = time.perf_counter() - t0
        kw_e = dict(kw, eliminate=True)
        re, (de, st) = rate(G, xt, yt, PL_PAIRS, 2, return_stats=True, **kw_e)
        _, st_plain = nvd.ge_distance(G, xt, yt, return_stats=True, **kw)
        de = de.cpu().numpy()
        ref = d2_ref.cpu().numpy()
        out["powerlaw_eliminated"] = {
            "distances_per_s": re, "elimination": info, "elimination_host_s": t_elim,
            "inner_iters_mean": float(np.mean([s_["iters"] for s_ in st])),
            "inner_iters_mean_plain": float(np.mean([s_["iters"] for s_ in st_plain])),
            "max_rel_diff_vs_plain": float(np.max(np.abs(de - ref) / np.abs(ref)))}
    return out


def run_er_large(args, nvd, synth, torch, np, rank, world, local, dist):
    """The Erdos-Renyi workload (n = 10^6, 8 pairs, one right-hand side at a time in
    FP64) as its own line, with the multi-RHS FP64 and MIXED comparisons."""
    dev = torch.device("cuda", local)
    wl = synth.workload_er_large()
    g = wl.graph
    X, Y = wl.pairs(*rank_pair_range(rank))                    # each rank its own pairs
    G = nvd.Graph.from_csr(g)
    # work decomposition picked by the autotuner on this graph (set-up, not timed)
    tuning = None if args.no_tune else G.tune(mode=nvd.MODE_FP64, k=PAIRS_PER_STEP, single_rhs=True)
    xt = torch.from_numpy(X).to(dev)
    yt = torch.from_numpy(Y).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        return nvd.ge_distance(G, xt, yt, rtol=RTOL, single_rhs=True, check_every=CHECK_EVERY,
                               return_stats=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    nvd.profile_enable(True, every=SPMV_SAMPLE)
    nvd.profile_read(0)
    nvd.profile_read(1)
    launches0 = nvd.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall0 = time.perf_counter()
    last = None
    for k in range(args.steps):
        flush.zero_()                                   # evict L2 between steps (not timed)
        ev[k][0].record()
        last = step()
        ev[k][1].record()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = nvd.kernel_launches() - launches0
    n_spmv, spmv_ms, spmv_bytes = nvd.profile_read(0)
    nvd.profile_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = job_time(sum(step_ms), dist, dev)
    d2_last, stats = last
    iters = [s["iters"] for s in stats]
    statuses = [s["status"] for s in stats]

    # ---- end to end through the C ABI with host buffers (copies inside the call)
    xh = torch.from_numpy(X).pin_memory()
    yh = torch.from_numpy(Y).pin_memory()
    for _ in range(2):
        nvd.ge_distance(G, xh, yh, rtol=RTOL, single_rhs=True, check_every=CHECK_EVERY)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    te0 = time.perf_counter()
    for _ in range(args.steps):
        d2_host = nvd.ge_distance(G, xh, yh, rtol=RTOL, single_rhs=True, check_every=CHECK_EVERY)
    torch.cuda.synchronize()
    te = job_time(time.perf_counter() - te0, dist, dev)

    # ---- the batched comparison the method is built for (same graph, same 8 pairs)
    extra = None
    if not args.no_extra and rank == 0:
        def rate(**kw):
            for _ in range(2):
                nvd.ge_distance(G, xt, yt, **kw)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            a.record()
            for _ in range(reps):
                out = nvd.ge_distance(G, xt, yt, **kw)
            b.record()
            torch.cuda.synchronize()
            return PAIRS_PER_STEP * reps / (a.elapsed_time(b) / 1e3), out
        # the accuracy the metric asks for (d^2 within 1e-6) reached by the d^2 stop
        # instead of the residual test (single-RHS tuning still in place)
        rsd, dsd = rate(rtol=1e-14, single_rhs=True, check_every=CHECK_EVERY, d2_stop=True, d2_rtol=D2_STOP_RTOL)
        _, st_sd = nvd.ge_distance(G, xt, yt, rtol=1e-14, single_rhs=True, check_every=CHECK_EVERY, d2_stop=True,
                                   d2_rtol=D2_STOP_RTOL, return_stats=True)
        tune64 = None if args.no_tune else G.tune(mode=nvd.MODE_FP64, k=PAIRS_PER_STEP)
        r64, d64 = rate(rtol=RTOL)
        rsdm, dsdm = rate(rtol=1e-14, d2_stop=True, d2_rtol=D2_STOP_RTOL)
        tunemx = None if args.no_tune else G.tune(mode=nvd.MODE_MIXED, k=PAIRS_PER_STEP)
        rmx, dmx = rate(mode=nvd.MODE_MIXED, rtol=MIXED_RTOL_IN, d2_rtol=MIXED_D2_RTOL)
        extra = {"fp64_multi_rhs_distances_per_s": r64, "mixed_multi_rhs_distances_per_s": rmx,
                 "mixed": f"FP32 block-PCG to rtol {MIXED_RTOL_IN} inside FP64 refinement to d2_rtol {MIXED_D2_RTOL}",
                 "tuning_fp64_multi": tune64, "tuning_mixed": tunemx,
                 "d2_fp64_multi": d64.cpu().numpy().tolist(), "d2_mixed": dmx.cpu().numpy().tolist(),
                 "d2stop": f"FP64 PCG stopped by the d^2 error estimate at d2_rtol {D2_STOP_RTOL} "
                           "(NVD_SOLVE_D2_STOP) instead of the residual test",
                 "fp64_single_rhs_d2stop_distances_per_s": rsd, "fp64_multi_rhs_d2stop_distances_per_s": rsdm,
                 "d2stop_iters_per_pair": [s_["iters"] for s_ in st_sd],
                 "d2_d2stop_single": dsd.cpu().numpy().tolist(), "d2_d2stop_multi": dsdm.cpu().numpy().tolist()}

    value = job_rate(PAIRS_PER_STEP, world, args.steps, total_ms)
    peaks, peak_src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    achieved = (spmv_bytes / n_spmv) / (spmv_ms / n_spmv / 1e3) / 1e9 if n_spmv else None
    folded = bool(tuning and tuning.get("fold_direction"))
    # the committed ncu traffic was taken on the three-kernel form's SpMV
    traffic = None if folded else ncu_traffic()
    kernel_name = ("k_spmm<double,double,double,1,EpiLapDir> (SpMV on D^-1 r, direction update folded in, p^T q)"
                   if folded else "k_spmm<double,double,double,1,EpiLap> (Laplacian SpMV + fused p^T q)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(g, wl.meta["n_generated"]), tuning=tuning),
        "e2e": {"value": job_rate(PAIRS_PER_STEP, world, args.steps, 1e3 * te), "unit": UNIT,
                "h2d_bytes_per_step": int(xh.numel() * 8 * 2), "d2h_bytes_per_step": PAIRS_PER_STEP * 8},
        "gpu_launches": int(launches),
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "kernel": kernel_name,
                     "launches": n_spmv, "sampled": f"1 in {SPMV_SAMPLE} SpMV launches of the timed steps",
                     "avg_launch_us": 1e3 * spmv_ms / n_spmv if n_spmv else None,
                     "algorithmic_bytes_per_launch": spmv_bytes / n_spmv if n_spmv else None,
                     "peak_source": f"{peak_src} hbm_gbs (STREAM-style copy) of MEASURED_PEAKS.json"},
        "solver": {"iters_per_pair": iters, "status": statuses, "wall_s_timed": t_wall,
                   "spmv_ms_per_step_est": spmv_ms * SPMV_SAMPLE / args.steps, "check_every": CHECK_EVERY},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, th, nsolves, dt, d2_or = cpu_baseline(g, X, Y)
        npairs = len(d2_or)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                                "sample": f"{nsolves} solves cycling over the step's {npairs} pairs ({dt:.1f} s), "
                                          f"oracle FP64 Jacobi-PCG (oracle/pcg.c) at rtol 1e-10"}
        got = d2_last.cpu().numpy()[:npairs]
        line["max_rel_err_vs_oracle"] = float(np.max(np.abs(got - d2_or) / np.abs(d2_or)))
        line["max_rel_err_e2e_vs_oracle"] = float(np.max(np.abs(d2_host.numpy()[:npairs] - d2_or)
                                                         / np.abs(d2_or)))
        if extra:
            extra["max_rel_err_fp64_multi"] = float(np.max(np.abs(np.array(extra["d2_fp64_multi"][:npairs])
                                                                  - d2_or) / np.abs(d2_or)))
            extra["max_rel_err_mixed"] = float(np.max(np.abs(np.array(extra["d2_mixed"][:npairs]) - d2_or)
                                                     / np.abs(d2_or)))
            for key in ("d2stop_single", "d2stop_multi"):
                extra["max_rel_err_" + key] = float(np.max(np.abs(np.array(extra["d2_" + key][:npairs]) - d2_or)
                                                          / np.abs(d2_or)))
    if extra:
        extra["multiple_mixed_vs_single_rhs_fp64"] = extra["mixed_multi_rhs_distances_per_s"] / value
        extra["multiple_fp64_multi_vs_single_rhs_fp64"] = extra["fp64_multi_rhs_distances_per_s"] / value
        extra["multiple_d2stop_single_vs_single_rhs_fp64"] = extra["fp64_single_rhs_d2stop_distances_per_s"] / value
        del extra["d2_fp64_multi"], extra["d2_mixed"], extra["d2_d2stop_single"], extra["d2_d2stop_multi"]
        line["batched_comparison"] = extra
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the multi-RHS comparison runs")
    ap.add_argument("--no-tune", action="store_true", help="default work decomposition (no autotuning)")
    ap.add_argument("--workload", choices=["er_large", "powerlaw", "batched", "grad", "resistance",
                                           "resistance_matrix"],
                    default="powerlaw",
                    help="powerlaw (default) is the bench line; the others measure the method's other workloads")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="--workload powerlaw: node-count multiplier (profiling runs on a smaller graph)")
    ap.add_argument("--tuning", default=None,
                    help="--workload powerlaw: JSON work decomposition applied with set_tuning instead of "
                         "autotuning, e.g. '{\"kt\": 16, \"row_max_pct\": 200}'")
    ap.add_argument("--eliminate", action="store_true",
                    help="--workload powerlaw: eliminate degree-1/2 nodes exactly and solve on the reduced graph")
    ap.add_argument("--sweep", choices=["size", "density"], default=None,
                    help="the paper's synthetic runtime sweeps (one GE per point) instead of the bench line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    import paper_2310_11222_gb300 as nvd
    import synth
    nvd.load_library()
    if args.sweep:
        return run_sweep(args, nvd, synth, torch, np, local)
    if args.workload == "powerlaw":
        return run_powerlaw(args, nvd, synth, torch, np, rank, world, local, dist)
    if args.workload == "er_large":
        return run_er_large(args, nvd, synth, torch, np, rank, world, local, dist)
    if world > 1:
        raise SystemExit("--workload other than powerlaw and er_large runs on one GPU")
    return run_other_workload(args, nvd, synth, torch, np, local)


if __name__ == "__main__":
    sys.exit(main())

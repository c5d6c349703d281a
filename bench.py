#!/usr/bin/env python
"""Benchmark: SAP-preconditioned FGMRES-DR solves of D x = b on one GB300.

One step = one complete solve (every stage of the path: SAP sweeps, the
Arnoldi product, Gram-Schmidt, Givens/least squares, deflated restarts and
the explicit residual) of the 16^3 x 32 Wilson workload: links
U = exp(i eps H) with eps = 0.5, bare mass putting the leftmost eigenvalue of
D at real part 1e-2, 4^4 domains, SAP 5 cycles x 4 MR steps, FGMRES-DR m = 30
k = 10, tol 1e-10, one Gaussian right-hand side. Inputs are resident in HBM
when the timed region starts (the Krylov working set, > 1 GB, exceeds L2).

The same JSON line carries the other workloads as legs: 12 right-hand sides
with FP16 SAP on the same lattice (the mixed-precision batched solver against
the plain one), the single-precision Arnoldi basis, FP64 outer vectors, the
clover operator, the stencil alone (GB/s against the measured HBM peak), the
SAP sweep's ALU roofline on three lattices, SAP as a stand-alone solver around
the spectral edge, the batched 24^3 x 48 point-source solve on the autotuned
block, the ill-conditioned 32^3 x 64 solve (FP16/BF16 SAP, FGMRES-DR(40,16)
against FGMRES(40)), the served Poisson stream (p50/p99 latency), the
conditioning of every workload, and the oracle's time for one complete solve
(cpu_baseline).

Prints one JSON line (rank 0). Under torchrun every rank solves its own
right-hand side (replicas; no data-path collective) and the timing is the
maximum over ranks. ``--impl reference`` times the FP64 CPU oracle on this
host's cores instead, in pieces of real solves of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D_w HBM GB/s & % roofline; SAP-FGMRES-DR solves/s, p50/p99 latency vs plain"
WORKLOAD = "wilson_16x16x16x32"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def workload():
    import fieldgen as fg

    cfg = dict(fg.lattice_configs()[WORKLOAD])
    return cfg


def sap_flops_per_site(block, nmr):
    """Algorithmic FP32 flops of one SAP colour sweep per swept site: the full
    stencil residual (1392) plus nmr MR steps on D^l (165 per in-domain hop,
    48 diagonal, 336 for the two inner products and two updates)."""
    hops_in = sum(2.0 * (b - 1) / b for b in block)
    return 1392.0 + nmr * (165.0 * hops_in + 48.0 + 336.0)


def kernel_traffic(name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    e = t.get(name)
    if not e:
        return None
    m = hashlib.sha256()
    for src in e["sources"]:
        m.update(open(os.path.join(ROOT, "paper_1204_5463_gb300", "csrc", src), "rb").read())
    if m.hexdigest()[:16] != e.get("source_sha256_16"):
        return None
    return e["bytes_per_launch"] * e.get("scale", 1.0)


def dw_bandwidth(peaks, reps=10, dims=(24, 24, 24, 48)):
    """The full-lattice stencil alone on a 24^3 x 48 lattice by default (its
    links and fields, 318 MB in FP32, exceed L2): algorithmic bytes per site (links +
    input + output: 960 B FP64, 480 B FP32, 248 B FP16 with scales) over the
    kernel's CUDA-event time, per storage precision. L2 is flushed (a 256 MB
    write) before every call; each call converts its input to the internal
    layout right before the stencil, so part of that input can still be in L2."""
    import numpy as np
    import torch

    import fieldgen as fg
    import paper_1204_5463_gb300 as dw

    dims = tuple(dims)
    U = fg.gauge_field(dims, 0.5, 0)
    psi = fg.gaussian_source(dims, 7)
    stream = torch.cuda.current_stream()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).reshape(-1).copy()).cuda()

    ctx = dw.dw_create(dims, (4, 4, 4, 4), -0.5, stream.cuda_stream)
    dw.dw_set_gauge(ctx, dev(U), True)
    ind = dev(psi)
    outd = torch.empty_like(ind)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"lattice": list(dims), "l2": "256 MB write before each call", "reps": reps}
    for name, prec in (("f64", dw.DW_F64), ("f32", dw.DW_F32), ("f16", dw.DW_F16)):
        torch.cuda.nvtx.range_push("dw_apply_" + name)  # lets a profiler select these launches
        dw.dw_apply(ctx, ind, outd, prec)  # builds this precision's link copy
        dw.dw_profile(ctx, True)
        dw.dw_profile_read(ctx, reset=True)
        for _ in range(reps):
            flush.zero_()
            dw.dw_apply(ctx, ind, outd, prec)
        torch.cuda.synchronize()
        d = dw.dw_profile_read(ctx, reset=True)["dw_" + name]
        dw.dw_profile(ctx, False)
        torch.cuda.nvtx.range_pop()
        avg_s = d["total_ms"] / d["launches"] / 1e3
        gbs = d["bytes"] / d["launches"] / avg_s / 1e9
        out[name] = {"GB/s": gbs, "frac": gbs / peaks["hbm_gbs"], "avg_us": avg_s * 1e6,
                     "bytes_per_site": d["bytes"] / d["launches"] / fg.volume(dims),
                     "Gsites_per_s": fg.volume(dims) / avg_s / 1e9,
                     "traffic": kernel_traffic("dw_" + name)}
    # 12 right-hand sides in one launch: the links count once per site for
    # all of them (FP32: (288 + 12 x 192) / 12 = 216 B per site and rhs,
    # FP16: (144 + 12 x 104) / 12 = 116 B); L2 serves the re-reads
    nb = 12
    psis = dev(fg.gaussian_source(dims, 8, nrhs=nb))
    outs = torch.empty_like(psis)
    for name, prec in (("f32", dw.DW_F32), ("f16", dw.DW_F16)):
        torch.cuda.nvtx.range_push("dw_apply_batched_" + name)
        dw.dw_apply(ctx, psis, outs, prec, nb)
        dw.dw_profile(ctx, True)
        dw.dw_profile_read(ctx, reset=True)
        for _ in range(reps):
            flush.zero_()
            dw.dw_apply(ctx, psis, outs, prec, nb)
        torch.cuda.synchronize()
        d = dw.dw_profile_read(ctx, reset=True)["dw_" + name]
        dw.dw_profile(ctx, False)
        torch.cuda.nvtx.range_pop()
        avg_s = d["total_ms"] / d["launches"] / 1e3
        gbs = d["bytes"] / d["launches"] / avg_s / 1e9
        out["batched_12rhs_" + name] = {"GB/s": gbs, "frac": gbs / peaks["hbm_gbs"], "avg_us": avg_s * 1e6,
                                        "us_per_rhs": avg_s * 1e6 / nb,
                                        "bytes_per_site_rhs": d["bytes"] / d["launches"] / fg.volume(dims) / nb,
                                        "Gsites_per_s": nb * fg.volume(dims) / avg_s / 1e9}
    dw.dw_destroy(ctx)
    return out


def oracle_kernels(cfg, U, b):
    """The oracle's D (GB/s at the FP64 algorithmic 960 B/site) and one SAP
    application (s cycles) on this workload, timed on the host cores."""
    import oracle

    V = 1
    for d in cfg["dims"]:
        V *= d
    oracle.dw(U, b, cfg["dims"], cfg["m0"])  # builds / loads the oracle
    t0 = time.perf_counter()
    oracle.dw(U, b, cfg["dims"], cfg["m0"])
    t_dw = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.sap(U, b, cfg["dims"], cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"])
    t_sap = time.perf_counter() - t0
    return {"dw_GB/s": 960.0 * V / t_dw / 1e9, "dw_s": t_dw, "sap_application_s": t_sap}


def oracle_solve_chunks(cfg, U, b):
    """A generator over a complete FP64 oracle solve of this workload
    (Algorithm 4 with the refinement of Sec. 5.7), one Arnoldi step per item."""
    import oracle

    A, M = oracle.lattice_operators(U, cfg["dims"], cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"])
    return oracle.fgmresdr_steps(A, M, b.reshape(-1), cfg["m"], cfg["k"], cfg["tol"])


def oracle_full_solve(cfg, U, b):
    """Seconds and Arnoldi steps of one complete oracle solve of this workload."""
    t0 = time.perf_counter()
    it = oracle_solve_chunks(cfg, U, b)
    steps = 0
    for _ in it:
        steps += 1
    return time.perf_counter() - t0, steps


def conditioning():
    """min |eigenvalue| of each workload's D at its bare mass (harmonic Ritz
    values of the oracle's D, stored with the spectral edges)."""
    import fieldgen as fg

    out = {}
    edges = fg.spectral_edges()
    for name, c in fg.lattice_configs().items():
        e = edges.get(fg.edge_key(c["dims"], c["eps"], c["seed"], c.get("csw", 0.0)))
        if not e or c.get("target_min_abs_eig") is None:
            continue
        ok = e.get("delta_ref") == c["target_min_abs_eig"]
        out[name] = {"delta": c["target_min_abs_eig"], "m0": c["m0"],
                     "min_abs_eig": e.get("min_abs_eig_at_m0_ref") if ok else None,
                     "method": e.get("method"), "converged": e.get("converged")}
    # the served fields at their smallest delta (1e-3)
    for d in ((8, 8, 8, 16), (16, 16, 16, 32), (24, 24, 24, 48)):
        for eps in (0.3, 0.6):
            e = edges.get(fg.edge_key(d, eps, 0), {})
            if e.get("method") == "harmonic_ritz":
                out[f"serving_{'x'.join(map(str, d))}_eps{eps}"] = {
                    "delta": e["delta_ref"], "m0": e["m0_ref"], "min_abs_eig": e["min_abs_eig_at_m0_ref"],
                    "method": e["method"], "converged": e["converged"]}
    return out


def max_over_ranks(values, dist=None, device="cuda"):
    """The maximum over all ranks of each value (a no-op without a process
    group): replica timings are taken as the slowest rank's."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def replica_throughput(units_per_rank, seconds, world):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle as it stands, on this host's
    cores, timed in pieces of real solves of the benchmark workload. Each step
    advances a running oracle solve by a fixed number of Arnoldi steps (with
    the cycle ends, deflated restarts and explicit residuals that fall in it);
    a solve that finishes is followed by a new one. solves/s = Arnoldi steps
    done / steps of a complete oracle solve / seconds; the step count of a
    complete solve is the one the timed region finished, else the stored
    count of the same solve (tests/golden)."""
    if rank != 0:
        return 0
    import fieldgen as fg

    cfg = workload()
    U = fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(cfg["dims"], 1)
    stored = stored_oracle_steps()
    n_est = stored or 80
    chunk = args.ref_chunk or max(1, -(-n_est // max(1, args.steps)))  # the K steps cover about one solve
    warm = oracle_solve_chunks(cfg, U, b)
    for _ in range(args.warmup):
        next(warm, None)
    del warm
    solve = oracle_solve_chunks(cfg, U, b)
    done_steps, finished, per = 0, [], []
    cur = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(chunk):
            if next(solve, None) is None:
                finished.append(cur)
                cur = 0
                solve = oracle_solve_chunks(cfg, U, b)
                if next(solve, None) is None:
                    break
            cur += 1
            done_steps += 1
        per.append(time.perf_counter() - t0)
    total = sum(per)
    steps_per_solve = finished[0] if finished else n_est
    value = done_steps / steps_per_solve / total
    sample = (f"{args.steps} pieces of {chunk} Arnoldi steps of a running FP64 oracle solve "
              f"({done_steps} steps, {len(finished)} solve(s) finished; {steps_per_solve} steps per solve, "
              + ("measured" if finished else "stored") + ")")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": cfg["dims"], "block": cfg["block"], "m0": cfg["m0"],
                   "m": cfg["m"], "k": cfg["k"], "sap": [cfg["sap_cycles"], cfg["mr_steps"]], "tol": cfg["tol"]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def stored_oracle_steps():
    """Arnoldi steps of the oracle's complete solve of the benchmark workload,
    as stored by tests/golden/make_golden.py (None when not stored for the
    current bare mass)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", WORKLOAD + "_oracle.json")) as f:
            g = json.load(f)
    except Exception:
        return None
    if abs(g["config"]["m0"] - workload()["m0"]) > 1e-12:
        return None
    return int(g["iterations"])


def _dev(a):
    import numpy as np
    import torch

    return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).reshape(-1).copy()).cuda()


_SERVING_FIELDS = {}


def serving_leg(args, rank, rate=None, window=None):
    """Continuous-batching serving of a Poisson stream of mixed solves.

    Requests: volumes uniform in {8^3x16, 16^3x32, 24^3x48}, eps in {0.3, 0.6},
    bare mass with the left spectral edge at delta ~ log-uniform[1e-3, 1e-2],
    1-12 Gaussian right-hand sides, tol 1e-10, FP16 SAP storage; arrivals
    Poisson at --rate req/s (seeded) over a fixed window of --window seconds;
    server budget 150 GB of device memory; latency = submit to done, drain
    included.
    """
    import threading

    import numpy as np

    import fieldgen as fg
    import paper_1204_5463_gb300 as dw

    rate = args.rate if rate is None else rate
    window = args.window if window is None else window
    rng = np.random.default_rng(1234 + rank)
    vols = [(8, 8, 8, 16), (16, 16, 16, 32), (24, 24, 24, 48)]
    epss = [0.3, 0.6]
    fields = {}
    for d in vols:
        for e in epss:  # generated once per process (both serving passes use them)
            if (d, e) not in _SERVING_FIELDS:
                _SERVING_FIELDS[(d, e)] = fg.gauge_field(d, e, seed=0)
            fields[(d, e)] = _SERVING_FIELDS[(d, e)]
    edges = fg.spectral_edges()
    reqs = []
    t = rng.exponential(1.0 / rate)
    i = 0
    while t < window:
        d = vols[rng.integers(len(vols))]
        e = epss[rng.integers(len(epss))]
        delta = float(np.exp(rng.uniform(np.log(1e-3), np.log(1e-2))))
        m0 = delta - edges[fg.edge_key(d, e, 0)]["edge_re"]
        nrhs = int(rng.integers(1, 13))
        b = np.ascontiguousarray(fg.gaussian_source(d, 5000 + i, nrhs=nrhs))
        reqs.append(dict(t=t, dims=d, eps=e, m0=m0, delta=delta, nrhs=nrhs, b=b, x=np.zeros_like(b)))
        t += rng.exponential(1.0 / rate)
        i += 1
    srv = dw.dw_server_create(int(150e9), args.slots)  # 150 GB budget
    keep = []
    ids = [None] * len(reqs)

    def submitter():
        t0 = time.perf_counter()
        for i, q in enumerate(reqs):
            dt = q["t"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            P = dw.dw_default_params(m=30, k=10, tol=1e-10, sap_cycles=5, mr_steps=4, sap_prec=dw.DW_F16,
                                     nrhs=q["nrhs"], outer_prec=dw.PREC[args.serving_outer])
            r = dw.make_request(q["dims"], (4, 4, 4, 4), q["m0"], fields[(q["dims"], q["eps"])], q["b"], q["x"], P)
            keep.append(r)
            ids[i] = dw.dw_server_submit(srv, r)

    t_start = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat, ok, solved = [], 0, 0
    for i, q in enumerate(reqs):
        status, S, l = dw.dw_server_wait(srv, ids[i], 3600)
        lat.append(l)
        ok += status == dw.DW_OK
        solved += S.converged
    wall = time.perf_counter() - t_start
    info = dw.dw_server_info(srv)
    dw.dw_server_destroy(srv)
    return {
        "metric": "served SAP-FGMRES-DR solves/s (continuous batching, HBM budget 150 GB)",
        "value": solved / wall, "unit": "solves/s", "requests": len(reqs), "requests_ok": ok,
        "rhs_solved": solved, "arrival_window_s": window, "offered_req_per_s": rate,
        "arrived_req_per_s": len(reqs) / window, "achieved_req_per_s": len(reqs) / wall, "wall_s": wall,
        "drain_s": wall - max(q["t"] for q in reqs) if reqs else 0.0,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "max": float(max(lat))},
        "peak_hbm_gb": info["peak_bytes"] / 1e9, "slots": args.slots, "peak_running": info["peak_running"],
        "dtype": "f16 SAP, f32 D z, " + ("FP32 Arnoldi basis with double-float residual" if args.serving_outer == "f32"
                                         else "double-float Arnoldi basis and residual"),
        "config": {"workload": "serving: volumes {8^3x16,16^3x32,24^3x48}, eps {0.3,0.6}, "
                               "leftmost eigenvalue at delta log-uniform [1e-3,1e-2], 1-12 rhs, tol 1e-10, m 30, "
                               "k 10, SAP 5x4"},
    }


def _profiled_sap(dw, torch, ctx, bd, ncyc, nmr, prec, nrhs, V, block):
    """Average SAP sweep of one preconditioner application (per-kernel events)."""
    zd = torch.empty_like(bd)
    dw.sap_precondition(ctx, bd, zd, ncyc, nmr, prec, nrhs)
    dw.dw_profile(ctx, True)
    dw.dw_profile_read(ctx, reset=True)
    for _ in range(3):
        dw.sap_precondition(ctx, bd, zd, ncyc, nmr, prec, nrhs)
    torch.cuda.synchronize()
    d = dw.dw_profile_read(ctx, reset=True)["sap_sweep"]
    dw.dw_profile(ctx, False)
    avg_s = d["total_ms"] / d["launches"] / 1e3
    flops = nrhs * (V / 2) * sap_flops_per_site(block, nmr)
    tf = flops / avg_s / 1e12
    # whole applications without per-kernel events (consecutive sweeps keep
    # their programmatic overlap): time per sweep, conversions included
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(3):
        dw.sap_precondition(ctx, bd, zd, ncyc, nmr, prec, nrhs)
    e1.record(st)
    torch.cuda.synchronize()
    app_s = e0.elapsed_time(e1) / 1e3 / (3 * 2 * ncyc)
    return {"nrhs": nrhs, "avg_us": avg_s * 1e6, "us_per_rhs": avg_s * 1e6 / nrhs, "achieved_tflops": tf,
            "frac": tf / FP32_PEAK_TFLOPS, "launches": d["launches"],
            "per_sweep_us_in_applications": app_s * 1e6,
            "frac_in_applications": flops / app_s / 1e12 / FP32_PEAK_TFLOPS}


def _solve_on(dw, torch, dims, block, m0, Ud, b, **kw):
    ctx = dw.dw_create(dims, block, m0, torch.cuda.current_stream().cuda_stream)
    try:
        dw.dw_set_gauge(ctx, Ud, True)
        P = dw.dw_default_params(**kw)
        bd = _dev(b)
        xd = torch.zeros_like(bd)
        dw.fgmresdr_solve(ctx, bd, xd, P, allow_notconv=True)  # warm-up: workspace and link copies
        xd.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = dw.fgmresdr_solve(ctx, bd, xd, P, allow_notconv=True)
        torch.cuda.synchronize()
        return S, time.perf_counter() - t0
    finally:
        dw.dw_destroy(ctx)


def mixed_leg(args):
    """The ill-conditioned 32^3 x 64 workload (leftmost eigenvalue of D at
    1e-3): FP16 and BF16 SAP storage, FGMRES-DR(40, 16) against restarted
    FGMRES(40) (capped at --k0-cycles cycles); and the FP32 SAP sweep alone on
    this lattice (its ALU roofline at 4096 domains per colour)."""
    import torch

    import fieldgen as fg
    import paper_1204_5463_gb300 as dw

    cfg = dict(fg.lattice_configs()["mixed_32x32x32x64"])
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    Ud = _dev(U)
    del U
    b = fg.gaussian_source(dims, 1)
    edges = fg.spectral_edges().get(fg.edge_key(dims, cfg["eps"], cfg["seed"]), {})
    out = {"lattice": list(dims), "m0": cfg["m0"], "eps": cfg["eps"], "delta": cfg["target_min_abs_eig"],
           "min_abs_eig": edges.get("min_abs_eig_at_m0_ref"), "runs": []}
    for prec, pname in ((dw.DW_F16, "f16"), (dw.DW_BF16, "bf16")):
        for k, cyc in ((cfg["k"], 400), (0, args.k0_cycles)):
            S, dt = _solve_on(dw, torch, dims, cfg["block"], cfg["m0"], Ud, b, m=cfg["m"], k=k, tol=cfg["tol"],
                              sap_cycles=cfg["sap_cycles"], mr_steps=cfg["mr_steps"], sap_prec=prec,
                              matvec_prec=dw.DW_F32, max_cycles=cyc)
            out["runs"].append({"sap_prec": pname, "m": cfg["m"], "k": k, "seconds": dt,
                                "converged": S.converged, "iterations": S.iterations, "cycles": S.cycles,
                                "clean_restarts": S.clean_restarts, "true_rel_res": S.true_rel_res[0]})
    ctx = dw.dw_create(dims, cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    dw.dw_set_gauge(ctx, Ud, True)
    out["sap_sweep_f32"] = _profiled_sap(dw, torch, ctx, _dev(b), cfg["sap_cycles"], cfg["mr_steps"], dw.DW_F32, 1,
                                         fg.volume(dims), cfg["block"])
    dw.dw_destroy(ctx)
    return out


def batched_leg(args):
    """The batched 24^3 x 48 workload: the 12 spin-colour point sources in one
    solve (FP16 SAP storage), on the domain block the autotuner picks by time
    to solution; and the FP32 SAP sweep alone on this lattice."""
    import torch

    import fieldgen as fg
    import paper_1204_5463_gb300 as dw

    cfg = dict(fg.lattice_configs()["batched_24x24x24x48"])
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    Ud = _dev(U)
    del U
    b = fg.point_sources(dims)
    out = {"lattice": list(dims), "m0": cfg["m0"], "eps": cfg["eps"], "delta": cfg["target_min_abs_eig"]}
    blk = tuple(cfg["block"])
    if not args.no_tune:
        bt, table = dw.dw_autotune_block(dims, cfg["m0"], Ud, _dev(b[:2]),
                                         dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=1e-6, sap_cycles=5,
                                                              mr_steps=4, nrhs=2, sap_prec=dw.DW_F16))
        out["autotune"] = {"best": bt, "candidates": [
            {"block": t[0], "seconds": t[1], "iterations": t[2], "status": t[3]} for t in table]}
        blk = bt
    S, dt = _solve_on(dw, torch, dims, blk, cfg["m0"], Ud, b, m=cfg["m"], k=cfg["k"], tol=cfg["tol"],
                      sap_cycles=cfg["sap_cycles"], mr_steps=cfg["mr_steps"], sap_prec=dw.DW_F16,
                      matvec_prec=dw.DW_F32, nrhs=12)
    out.update({"block": list(blk), "nrhs": 12, "sap_prec": "f16", "seconds": dt, "value": S.converged / dt,
                "unit": "solves/s", "converged": S.converged, "iterations_max": S.iterations, "cycles": S.cycles,
                "true_rel_res_max": max(S.true_rel_res[i] for i in range(12))})
    ctx = dw.dw_create(dims, cfg["block"], cfg["m0"], torch.cuda.current_stream().cuda_stream)
    dw.dw_set_gauge(ctx, Ud, True)
    out["sap_sweep_f32"] = _profiled_sap(dw, torch, ctx, _dev(fg.gaussian_source(dims, 1)), cfg["sap_cycles"],
                                         cfg["mr_steps"], dw.DW_F32, 1, fg.volume(dims), cfg["block"])
    dw.dw_destroy(ctx)
    return out


def sap_standalone_leg(args, cfg, Ud):
    """SAP as a stand-alone solver (Sec. 3; the analogue of Fig. 5): the
    relative residual after s cycles from x = 0 on the benchmark lattice, for
    bare masses around the spectral edge of D (delta = leftmost real part of
    spec D_m0)."""
    import torch

    import fieldgen as fg
    import paper_1204_5463_gb300 as dw

    dims = cfg["dims"]
    edge = fg.spectral_edges()[fg.edge_key(dims, cfg["eps"], cfg["seed"])]["edge_re"]
    bd = _dev(fg.gaussian_source(dims, 1))
    zd = torch.empty_like(bd)
    rd = torch.empty_like(bd)
    out = {"lattice": list(dims), "sap_cycles_max": args.sap_cycles_max, "mr_steps": cfg["mr_steps"], "runs": []}
    for delta in (0.3, 0.1, 0.03, 0.01, -0.01, -0.03, -0.1):
        m0 = delta - edge
        ctx = dw.dw_create(dims, cfg["block"], m0, torch.cuda.current_stream().cuda_stream)
        try:
            dw.dw_set_gauge(ctx, Ud, True)
            hist = []
            for s_ in range(1, args.sap_cycles_max + 1):
                dw.sap_precondition(ctx, bd, zd, s_, cfg["mr_steps"], dw.DW_F32, 1)
                dw.dw_apply(ctx, zd, rd, dw.DW_F64, 1)
                hist.append(float(torch.linalg.vector_norm(bd - rd) / torch.linalg.vector_norm(bd)))
        finally:
            dw.dw_destroy(ctx)
        best = min(range(len(hist)), key=lambda i: hist[i])
        out["runs"].append({"delta": delta, "m0": m0, "kappa": 1.0 / (2.0 * (4.0 + m0)),
                            "rel_res_by_cycle": [round(h, 9) for h in hist], "min_at_cycle": best + 1,
                            "diverges": hist[-1] > 2 * hist[best]})
    return out


def run_workload(args, rank, world):
    """One extra leg alone (--workload batched_24x24x24x48, mixed_32x32x32x64 or
    sap_standalone, or --serving), printed as its own JSON line."""
    import torch

    import fieldgen as fg

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.serving:
        out = serving_leg(args, rank)
    elif args.workload == "sap_standalone":
        cfg = workload()
        out = sap_standalone_leg(args, cfg, _dev(fg.gauge_field(cfg["dims"], cfg["eps"], cfg["seed"])))
    elif args.workload == "sap_sweep":
        # the SAP sweep alone (FP32, one rhs, the benchmark's SAP settings) on
        # the lattice of --dw-lattice: its ALU roofline where the grid fills the GPU
        import paper_1204_5463_gb300 as dw

        dims = tuple(int(v) for v in args.dw_lattice.split("x"))
        ctx = dw.dw_create(dims, (4, 4, 4, 4), -0.6, torch.cuda.current_stream().cuda_stream)
        dw.dw_set_gauge(ctx, _dev(fg.gauge_field(dims, 0.5, 0)), True)
        out = {"workload": "sap_sweep", "lattice": list(dims),
               "sap_sweep_f32": _profiled_sap(dw, torch, ctx, _dev(fg.gaussian_source(dims, 1)), 5, 4, dw.DW_F32, 1,
                                              fg.volume(dims), (4, 4, 4, 4))}
        dw.dw_destroy(ctx)
    elif args.workload.startswith("batched"):
        out = batched_leg(args)
    elif args.workload.startswith("mixed"):
        out = mixed_leg(args)
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-chunk", type=int, default=0,
                    help="Arnoldi steps of the oracle per reference-arm step (0: the K steps cover one solve)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the legs of the other workloads (mixed 32^3x64, batched 24^3x48, serving, "
                         "stand-alone SAP)")
    ap.add_argument("--sap-prec", default="f32")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-dw-bw", action="store_true", help="skip the stand-alone D_w bandwidth measurement")
    ap.add_argument("--dw-lattice", default="24x24x24x48", help="lattice of the stand-alone D_w measurement")
    ap.add_argument("--serving", action="store_true", help="run the serving measurement instead")
    ap.add_argument("--window", type=float, default=0.8, help="arrival window of the served Poisson stream (s)")
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--stable-rate", type=float, default=0.5, help="offered rate of the sustained serving pass")
    ap.add_argument("--stable-window", type=float, default=20.0, help="arrival window of the sustained pass (s)")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serving-outer", default="df64", choices=["df64", "f32"],
                    help="Arnoldi basis of the served solves (f32: the single-precision scheme of Sec. 5.7)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="wilson_16x16x16x32 (default, the benchmark line), batched_24x24x24x48, mixed_32x32x32x64, "
                         "sap_standalone (SAP as a solver around the spectral edge, 16^3x32), sap_sweep (one SAP "
                         "application alone on --dw-lattice)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--k0-cycles", type=int, default=40, help="cycle cap of the restarted FGMRES comparison")
    ap.add_argument("--sap-cycles-max", type=int, default=30, help="SAP cycles of the stand-alone SAP runs")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        if args.impl == "ours":
            torch.cuda.set_device(local)
        # the reference arm runs the CPU oracle: gloo, no device
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.serving or args.workload != WORKLOAD:
        return run_workload(args, rank, world)
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return rc

    import fieldgen as fg
    import paper_1204_5463_gb300 as dw

    torch.cuda.set_device(local)
    cfg = workload()
    dims, block = cfg["dims"], cfg["block"]
    V = fg.volume(dims)
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(dims, 1 + rank)
    stream = torch.cuda.current_stream()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.float64).reshape(-1).copy()).cuda()

    ctx = dw.dw_create(dims, block, cfg["m0"], stream.cuda_stream)
    Ud = dev(U)
    dw.dw_set_gauge(ctx, Ud, True)
    bd = dev(b)
    xd = torch.zeros_like(bd)
    P = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                             mr_steps=cfg["mr_steps"], sap_prec=dw.PREC[args.sap_prec], matvec_prec=dw.DW_F32)

    for _ in range(args.warmup):
        S = dw.fgmresdr_solve(ctx, bd, xd, P)
    torch.cuda.synchronize()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    barrier()
    if clocks:
        clocks.start()
    # timed region 1: K solves as a user runs them (no per-kernel events)
    launches0 = dw.dw_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    lat = []
    iters = []
    cleans = []
    ev0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        S = dw.fgmresdr_solve(ctx, bd, xd, P)
        lat.append(1e3 * (time.perf_counter() - t0))
        iters.append(S.iterations)
        cleans.append(S.clean_restarts)
        assert S.converged == 1 and S.true_rel_res[0] <= cfg["tol"]
    ev1.record(stream)
    barrier()
    launches = dw.dw_kernel_launches() - launches0
    # residual against Arnoldi steps per cycle of the last timed solve (the paper's plots)
    history = [[h[0], h[1], h[2]] for h in dw.dw_residual_history(ctx, 0)]
    # timed region 2: the same K solves with the library's per-kernel CUDA
    # events on the solver's stream (the roofline and the kernel shares); the
    # events themselves cost wall time, so the headline comes from region 1
    dw.dw_profile(ctx, True)
    dw.dw_profile_read(ctx, reset=True)
    barrier()
    pe0 = torch.cuda.Event(enable_timing=True)
    pe1 = torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        S = dw.fgmresdr_solve(ctx, bd, xd, P)
        assert S.converged == 1 and S.true_rel_res[0] <= cfg["tol"]
    pe1.record(stream)
    barrier()
    clk = clocks.stop() if clocks else None
    prof = dw.dw_profile_read(ctx, reset=True)
    dw.dw_profile(ctx, False)
    ms_prof = pe0.elapsed_time(pe1)
    ms = ev0.elapsed_time(ev1)
    ms, ms_prof = max_over_ranks([ms, ms_prof], dist)
    value = replica_throughput(args.steps, ms / 1e3, world)

    # end to end through the C ABI with host buffers (pinned), copies inside the call
    bh = torch.from_numpy(np.ascontiguousarray(b).view(np.float64).reshape(-1).copy()).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    Ph = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                              mr_steps=cfg["mr_steps"], sap_prec=dw.PREC[args.sap_prec], matvec_prec=dw.DW_F32,
                              host_buffers=1)
    dw.fgmresdr_solve(ctx, bh.data_ptr(), xh.data_ptr(), Ph)
    barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        dw.fgmresdr_solve(ctx, bh.data_ptr(), xh.data_ptr(), Ph)
    barrier()
    e2e_s = time.perf_counter() - e0
    (e2e_s,) = max_over_ranks([e2e_s], dist)
    e2e_value = replica_throughput(args.steps, e2e_s, world)

    # the same lattice, 12 right-hand sides per launch, FP16 SAP storage: the
    # mixed-precision batched solver against the plain single-rhs one above
    mb = None
    if not args.no_batched:
        b12 = fg.gaussian_source(dims, 100 + rank, nrhs=12)
        b12d = dev(b12)
        x12d = torch.zeros_like(b12d)
        P12 = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                   mr_steps=cfg["mr_steps"], sap_prec=dw.DW_F16, matvec_prec=dw.DW_F32, nrhs=12)
        S12 = dw.fgmresdr_solve(ctx, b12d, x12d, P12)
        barrier()
        m0e, m1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0e.record(stream)
        nb_steps = max(1, args.steps // 2)
        for _ in range(nb_steps):
            S12 = dw.fgmresdr_solve(ctx, b12d, x12d, P12)
            assert S12.converged == 12
        m1e.record(stream)
        barrier()
        (mms,) = max_over_ranks([m0e.elapsed_time(m1e)], dist)
        mb_value = replica_throughput(12 * nb_steps, mms / 1e3, world)
        mb = {"value": mb_value, "unit": "solves/s", "nrhs": 12, "sap_prec": "f16", "steps": nb_steps,
              "ms_per_step": mms / nb_steps, "iterations_max": S12.iterations,
              "true_rel_res_max": max(S12.true_rel_res[i] for i in range(12)), "ratio_vs_plain": mb_value / value}
        # the same with the single-precision Arnoldi basis of Sec. 5.7 (refined per cycle)
        P12s = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                    mr_steps=cfg["mr_steps"], sap_prec=dw.DW_F16, matvec_prec=dw.DW_F32, nrhs=12,
                                    outer_prec=dw.DW_F32)
        S12 = dw.fgmresdr_solve(ctx, b12d, x12d, P12s)
        barrier()
        m0e.record(stream)
        for _ in range(nb_steps):
            S12 = dw.fgmresdr_solve(ctx, b12d, x12d, P12s)
            assert S12.converged == 12
        m1e.record(stream)
        barrier()
        (mms,) = max_over_ranks([m0e.elapsed_time(m1e)], dist)
        v2 = replica_throughput(12 * nb_steps, mms / 1e3, world)
        mb["f32_basis"] = {"value": v2, "unit": "solves/s", "ms_per_step": mms / nb_steps,
                           "iterations_max": S12.iterations,
                           "true_rel_res_max": max(S12.true_rel_res[i] for i in range(12)),
                           "ratio_vs_plain": v2 / value}
        # SAP cycles and MR steps tuned for this batched FP16 setting (time to
        # solution of a calibration solve per pair), both basis formats
        for label, outer in (("tuned_sap", dw.DW_DF64), ("tuned_sap_f32_basis", dw.DW_F32)):
            Pt = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_prec=dw.DW_F16,
                                      matvec_prec=dw.DW_F32, nrhs=12, outer_prec=outer)
            (tc, tm), ttab = dw.dw_autotune_sap(dims, block, cfg["m0"], Ud, b12d, Pt)
            Pt.sap_cycles, Pt.mr_steps = tc, tm
            S12 = dw.fgmresdr_solve(ctx, b12d, x12d, Pt)
            barrier()
            m0e.record(stream)
            for _ in range(nb_steps):
                S12 = dw.fgmresdr_solve(ctx, b12d, x12d, Pt)
                assert S12.converged == 12
            m1e.record(stream)
            barrier()
            (mms,) = max_over_ranks([m0e.elapsed_time(m1e)], dist)
            vt = replica_throughput(12 * nb_steps, mms / 1e3, world)
            mb[label] = {"value": vt, "unit": "solves/s", "sap": [tc, tm], "ms_per_step": mms / nb_steps,
                         "iterations_max": S12.iterations,
                         "true_rel_res_max": max(S12.true_rel_res[i] for i in range(12)),
                         "ratio_vs_plain": vt / value,
                         "calibration": [{"sap": [t[0], t[1]], "seconds": round(t[2], 4), "iterations": t[3]}
                                         for t in ttab if t[4] == dw.DW_OK]}
        del b12d, x12d

    # the paper's single-precision Arnoldi process with double-float refinement
    # per cycle (FP32 basis), same lattice, rhs and solver parameters
    sp32 = None
    if not args.no_batched:
        P32 = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                   mr_steps=cfg["mr_steps"], sap_prec=dw.PREC[args.sap_prec], matvec_prec=dw.DW_F32,
                                   outer_prec=dw.DW_F32)
        S32 = dw.fgmresdr_solve(ctx, bd, xd, P32)
        barrier()
        s0e, s1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0e.record(stream)
        for _ in range(args.steps):
            S32 = dw.fgmresdr_solve(ctx, bd, xd, P32)
            assert S32.converged == 1 and S32.true_rel_res[0] <= cfg["tol"]
        s1e.record(stream)
        barrier()
        (sms,) = max_over_ranks([s0e.elapsed_time(s1e)], dist)
        sv = replica_throughput(args.steps, sms / 1e3, world)
        sp32 = {"value": sv, "unit": "solves/s", "outer_prec": "f32 basis, double-float x/b/r",
                "ms_per_step": sms / args.steps, "iterations": S32.iterations, "cycles": S32.cycles,
                "clean_restarts": S32.clean_restarts, "true_rel_res": S32.true_rel_res[0],
                "ratio_vs_plain": sv / value}

    # FP64 outer vectors (the Arnoldi basis, x, b, r and their Gram-Schmidt in
    # native FP64) beside the double-float headline, same lattice and rhs
    f64o = None
    if not args.no_batched:
        P64 = dw.dw_default_params(m=cfg["m"], k=cfg["k"], tol=cfg["tol"], sap_cycles=cfg["sap_cycles"],
                                   mr_steps=cfg["mr_steps"], sap_prec=dw.PREC[args.sap_prec], matvec_prec=dw.DW_F32,
                                   outer_prec=dw.DW_F64)
        S64 = dw.fgmresdr_solve(ctx, bd, xd, P64)
        barrier()
        f0e, f1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0e.record(stream)
        for _ in range(args.steps):
            S64 = dw.fgmresdr_solve(ctx, bd, xd, P64)
            assert S64.converged == 1 and S64.true_rel_res[0] <= cfg["tol"]
        f1e.record(stream)
        barrier()
        (fms,) = max_over_ranks([f0e.elapsed_time(f1e)], dist)
        fv = replica_throughput(args.steps, fms / 1e3, world)
        f64o = {"value": fv, "unit": "solves/s", "outer_prec": "f64 basis, x, b, r",
                "ms_per_step": fms / args.steps, "iterations": S64.iterations, "cycles": S64.cycles,
                "clean_restarts": S64.clean_restarts, "true_rel_res": S64.true_rel_res[0],
                "ratio_vs_double_float": fv / value}
        if mb:
            # the mixed-precision batched variants against the plain solver as
            # the workload defines it (FP32 stencil, FP64 outer vectors) as well
            for leg in [mb] + [mb[k] for k in ("f32_basis", "tuned_sap", "tuned_sap_f32_basis") if k in mb]:
                leg["ratio_vs_plain_fp64_outer"] = leg["value"] / fv

    # the clover-improved operator (c_sw = 1.91, the paper's 16^3 x 32 value)
    # on the same links, bare mass tuned to its own spectral edge
    clov = None
    ccfg = fg.lattice_configs().get("clover_16x16x16x32")
    if not args.no_batched and ccfg and ccfg["m0"] is not None:
        cctx = dw.dw_create(dims, block, ccfg["m0"], stream.cuda_stream)
        dw.dw_set_gauge(cctx, Ud, True)
        dw.dw_set_clover(cctx, ccfg["csw"])
        Pc = dw.dw_default_params(m=ccfg["m"], k=ccfg["k"], tol=ccfg["tol"], sap_cycles=ccfg["sap_cycles"],
                                  mr_steps=ccfg["mr_steps"], sap_prec=dw.PREC[args.sap_prec], matvec_prec=dw.DW_F32)
        Sc = dw.fgmresdr_solve(cctx, bd, xd, Pc)
        barrier()
        c0e, c1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0e.record(stream)
        for _ in range(args.steps):
            Sc = dw.fgmresdr_solve(cctx, bd, xd, Pc)
            assert Sc.converged == 1 and Sc.true_rel_res[0] <= ccfg["tol"]
        c1e.record(stream)
        barrier()
        (cms,) = max_over_ranks([c0e.elapsed_time(c1e)], dist)
        cv = replica_throughput(args.steps, cms / 1e3, world)
        clov = {"value": cv, "unit": "solves/s", "csw": ccfg["csw"], "m0": ccfg["m0"],
                "ms_per_step": cms / args.steps, "iterations": Sc.iterations, "cycles": Sc.cycles,
                "clean_restarts": Sc.clean_restarts, "true_rel_res": Sc.true_rel_res[0]}
        dw.dw_destroy(cctx)

    # roofline of the dominant kernel class of the step
    peaks, peak_src = measured_peaks()
    dom = max(prof, key=lambda k: prof[k]["total_ms"])
    d = prof[dom]
    avg_ms = d["total_ms"] / d["launches"]
    if dom == "sap_sweep":
        flops = (V / 2) * sap_flops_per_site(block, cfg["mr_steps"])
        achieved = flops / (avg_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP32_PEAK_TFLOPS, "peak_source": "derived (152 SM x 128 FP32 x 2 x 2.07 GHz)"}
        # the same launches against HBM (algorithmic bytes: links, v, x read and x written per swept site)
        gbs = (d["bytes"] / d["launches"]) / (avg_ms / 1e3) / 1e9
        roof["hbm"] = {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                       "peak_source": peak_src}
    else:
        achieved = (d["bytes"] / d["launches"]) / (avg_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_src}
    tr = kernel_traffic(dom)
    roof.update({"kernel": dom, "traffic": tr, "launches": d["launches"], "avg_us": 1e3 * avg_ms})
    shares = {k: round(v["total_ms"] / sum(x["total_ms"] for x in prof.values()), 4) for k, v in prof.items()}
    avg_us = {k: round(1e3 * v["total_ms"] / v["launches"], 2) for k, v in prof.items() if v["launches"]}
    dwbw = None if args.no_dw_bw else dw_bandwidth(peaks, dims=tuple(int(v) for v in args.dw_lattice.split("x")))
    sap16 = _profiled_sap(dw, torch, ctx, bd, cfg["sap_cycles"], cfg["mr_steps"], dw.DW_F32, 1, V, block)
    extra = {}
    if not args.no_extra and world == 1:  # single-GPU workloads, measured at N = 1 only
        extra["sap_standalone"] = sap_standalone_leg(args, cfg, Ud)
        extra["batched_24x24x24x48"] = batched_leg(args)
        extra["mixed_32x32x32x64"] = mixed_leg(args)
        extra["serving"] = serving_leg(args, rank)
        # the same stream at a rate the GPU sustains: latency without a growing queue
        extra["serving"]["sustained"] = serving_leg(args, rank, rate=args.stable_rate, window=args.stable_window)

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 SAP and D z, double-float Arnoldi basis and residual", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(dims), "block": list(block), "m0": cfg["m0"],
                   "eps": cfg["eps"], "m": cfg["m"], "k": cfg["k"], "sap": [cfg["sap_cycles"], cfg["mr_steps"]],
                   "sap_prec": args.sap_prec, "tol": cfg["tol"], "nrhs": 1, "parallelism": f"replicas x{world}",
                   "l2": "working set > L2 (Krylov basis ~0.8 GB)"},
        "latency_ms": {"p50": statistics.median(lat), "p99": float(np.percentile(lat, 99)), "min": min(lat)},
        "iterations": iters,
        "clean_restarts": cleans,
        "residual_history": {"columns": ["arnoldi_steps", "implicit_rel_res", "explicit_rel_res"],
                             "cycles": history},
        "roofline": roof,
        "kernel_share": shares,
        "kernel_avg_us": avg_us,
        "profiled_pass": {"ms_per_step": ms_prof / args.steps, "steps": args.steps,
                          "note": "second timed pass with per-kernel CUDA events (roofline, kernel_share, "
                                  "kernel_avg_us); value is the pass without them"},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(bh.numel() * 8),
                "d2h_bytes_per_step": int(xh.numel() * 8)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "mixed_batched": mb,
        "fp32_arnoldi": sp32,
        "fp64_outer": f64o,
        "clover": clov,
        "dw_apply": dwbw,
        "sap_sweep_by_lattice": {"16x16x16x32": sap16,
                                 "24x24x24x48": extra.get("batched_24x24x24x48", {}).get("sap_sweep_f32"),
                                 "32x32x32x64": extra.get("mixed_32x32x32x64", {}).get("sap_sweep_f32")},
        "conditioning": conditioning(),
        **extra,
    }
    if rank == 0 and not args.no_cpu_baseline:
        secs, n = oracle_full_solve(cfg, U, b)
        line["cpu_baseline"] = {"value": 1.0 / secs, "unit": "solves/s", "cores": cores(), "kind": "oracle",
                                "sample": f"one complete FP64 oracle solve of this workload ({n} Arnoldi steps, "
                                          f"{secs:.1f} s)",
                                "kernels": oracle_kernels(cfg, U, b)}
    dw.dw_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

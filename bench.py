#!/usr/bin/env python
"""Benchmark of the Kernel-SDF back-end hot path on GB300 (one JSON line on rank 0).

One step = the whole path over one batch of the scale workload (50 x 50 x 10 m scene with 1,000 spheres
and boxes, 2,000,000 noisy surface samples, 0.5 m cells capped at 512 samples, a 256^3 grid of
16,777,216 queries): the fit of every local GP (binning, cell index, training sets, FP64 Cholesky / alpha,
FP32 L^-1), the query (candidates, min-fused SDF, gradient, softmin variance, GP variance) and the adjoint
of sdf and grad with respect to the query points and the sample positions.  value = queries per second
of that step over all ranks (weak scaling: each rank fits the scene and answers its own batch).  Inputs
are resident on the device; L2 (129 MB) is flushed with a 256 MiB write between timed steps.

The JSON line also carries: the roofline of the query and its adjoint (the binding unit among MUFU, FP32,
tensor cores and HBM, from algorithmic counts of this run's model and queries, against peaks measured
live by the probes of libksdf_peaks.so), the per-kernel rooflines and stage times, the plain FP64 GPU
query of the same inputs, the end-to-end rate through the C ABI with pinned host buffers, the CPU FP64
oracle on a bounded sample (cpu_baseline) with a parity check of this run's outputs on that sample, SM
clocks sampled during the timed region, the number of kernel launches, and the other workloads.  Among them,
city_frontend runs the BHM front-end (Sec. IV-A) over the city stream's 100 LiDAR frames (update, surface
points, sign), and its pipeline the paper's per-frame data flow with a persistent GP map: the BHM's surface
points replace the re-marched ones in the GPs, and the SDF query is signed by the BHM.

--impl reference times the CPU FP64 oracle itself (the reference arm; the paper ships no implementation
to run) with the same per-step protocol as cpu_baseline.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "scale3d_query_adjoint_dram.txt")
METRIC = "SDF+grad+var queries/s at err<=1e-4 m vs FP64 oracle; % roofline; vs plain FP64"
CITY_REFIT_BUDGET = 2000  # cells refitted per frame in the scheduled city stream
WORKLOAD_TEXT = {
    "scale3d": ("scale3d: 50x50x10 m scene with 1,000 spheres/boxes, 2,000,000 samples (sigma 0.01 m), 0.5 m cells, "
                "n_max 512, K 8, lambda 300; 256^3 = 16,777,216 grid queries; step = fit + query(sdf, grad, var_sdf, "
                "var_f) + adjoint(d sdf, d grad -> d xq, d x)"),
    "room3d": ("room3d: 20x20x5 m room with 50 spheres/boxes, 200,000 samples (sigma 0.01 m), 0.5 m cells, n_max 256, "
               "K 8, lambda 300; 1,000,000 uniform queries; step = fit + query(sdf, grad, var_sdf, var_f) + "
               "adjoint(d sdf, d grad -> d xq, d x)"),
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale3d", choices=sorted(WORKLOAD_TEXT))
    ap.add_argument("--samples", type=int, default=None, help="override the workload's sample count (tests)")
    ap.add_argument("--queries", type=int, default=None, help="override the workload's query count (tests)")
    ap.add_argument("--cpu-sample", type=int, default=65536, help="queries of the oracle's per-step sample")
    ap.add_argument("--cpu-repeats", type=int, default=3, help="oracle steps of the cpu_baseline leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle leg (cpu_baseline, parity)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-graph", action="store_true", help="launch query + adjoint eagerly instead of a CUDA graph")
    return ap.parse_args(argv)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def whole_job_rate(total_s, world, queries_per_rank, steps, device=None):
    """The slowest rank's timed seconds (all-reduce MAX over the ranks) and the whole job's queries/s: every
    rank answers its own batch (weak scaling), so the job's rate is world x batch x steps over that time."""
    if world > 1:
        import torch
        import torch.distributed as dist

        tt = torch.tensor([total_s], device=device, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_s = float(tt.item())
    return total_s, world * queries_per_rank * steps / total_s


def make_workload(args, rank):
    """The benchmark workload; rank 0 answers the workload's own queries, every other rank the same number of
    seeded uniform queries in the scene's box (its own batch of the same scene)."""
    from paper_2603_29227_gb300 import scenes

    name = getattr(args, "workload", None) or "scale3d"
    nq = getattr(args, "queries", None)
    if name == "scale3d":
        grid = None if nq is None else max(2, int(round(nq ** (1.0 / 3.0))))
        w = scenes.workload("scale3d", n_samples=getattr(args, "samples", None), grid=grid)
    else:
        w = scenes.workload(name, n_samples=getattr(args, "samples", None), n_queries=nq)
    if rank > 0:
        rng = np.random.default_rng(1000 + rank)
        lo, hi = w.scene.room_lo, w.scene.room_hi
        w.xq = np.ascontiguousarray(lo + rng.random((len(w.xq), 3)) * (hi - lo), dtype=np.float32)
        w.sign = w.scene.sign(w.xq.astype(np.float64))
    return w


def workload_config(w, args):
    """The config block shared by both arms (same keys, same values)."""
    return {"workload": WORKLOAD_TEXT[w.name], "samples": int(len(w.x)), "queries": int(len(w.xq)),
            "l2": "inputs resident in HBM; L2 flushed between timed steps (256 MiB write outside the step events)"}


# ----------------------------------------------------------------------------------------------------
# CPU FP64 oracle: the same per-step protocol for the reference arm and cpu_baseline


def oracle_step(w, sel, d_sdf, d_grad):
    """One oracle step: the full FP64 fit of every sample and the forward + adjoint of the queries `sel`.
    Returns (fit seconds, query+adjoint seconds, forward outputs on sel)."""
    import oracle

    t0 = time.perf_counter()
    m = oracle.Model(w.params, w.x, w.var, w.normals)
    t1 = time.perf_counter()
    ref = m.query(w.xq[sel], w.sign[sel], with_cands=True)
    m.backward(w.xq[sel], d_sdf, d_grad, sign=w.sign[sel], winner=ref["winner"])
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, ref, m


def oracle_sample(w, n_sample, seed=0):
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(w.xq), size=min(n_sample, len(w.xq)), replace=False))
    d_sdf = np.ones(len(sel))
    d_grad = np.random.default_rng(7).standard_normal((len(sel), w.params["dim"])) * 0.1
    return sel, d_sdf, d_grad


def oracle_stats(w, sel, fit_s, qb_s, threads):
    """cpu_baseline block: value = the sample's queries per second of measured step time (fit included);
    the whole-workload rate the same oracle would reach (one fit per full batch) is a separate field."""
    q, Q = len(sel), len(w.xq)
    fit_m, qb_m = float(np.mean(fit_s)), float(np.mean(qb_s))
    return {"value": q / (fit_m + qb_m), "unit": "queries/s", "cores": threads, "kind": "oracle",
            "sample": "per step: the full FP64 fit of all %d samples + forward and adjoint of %d seeded random queries "
                      "of the %d (no scaling); %d steps" % (len(w.x), q, Q, len(fit_s)),
            "ms_per_step": 1e3 * (fit_m + qb_m), "fit_s": fit_m, "query_adjoint_s": qb_m,
            "extrapolated_full_workload_rate": Q / (fit_m + qb_m * Q / q),
            "extrapolated_how": "one fit + the sample's per-query time x all queries of the workload"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    w = make_workload(args, 0)
    oracle.build()
    threads = oracle.set_threads(os.cpu_count() or 1)
    sel, d_sdf, d_grad = oracle_sample(w, args.cpu_sample)
    fit_s, qb_s = [], []
    for it in range(args.warmup + args.steps):
        tf, tq, _, m = oracle_step(w, sel, d_sdf, d_grad)
        del m
        if it >= args.warmup:
            fit_s.append(tf)
            qb_s.append(tq)
    cpu = oracle_stats(w, sel, fit_s, qb_s, threads)
    value = cpu["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cpu["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args), "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------------
# clocks


class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        rows = [ln.split(", ") for ln in self.lines if ln]
        mine = [r for r in rows if self.uuid and r[0].strip() == self.uuid] or rows
        if not mine:
            return None
        sm = [float(r[1]) for r in mine if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in mine if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in mine:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(mine)}


# ----------------------------------------------------------------------------------------------------
# algorithmic work (roofline numerators)


def fit_fp64_flops(n):
    """FP64 flops of the factorisation stage (k_fit) for cells with training-set sizes n: Cholesky N^3/3 and
    alpha 2N^2 (two triangular solves)."""
    n = n.astype(np.float64)
    return float(np.sum(n ** 3 / 3 + 2 * n ** 2))


def query_work(w, h, winner):
    """Algorithmic counts of the query and of its adjoint on this model and batch.  Per query, C = sum of the
    candidate cells' training-set sizes and N_w = the winner's:
      forward   MUFU  C (phase A exp) + 3 N_w (k', z, softmin weight) + 3;   FP32 lane ops 8 C + 18 N_w;
                V[f]: N_w (N_w + 1) / 2 MACs of K' L^-T, on the tensor cores (N_w <= 256) as TF32 split three
                ways, 3 N_w (N_w + 1) flops, else N_w (N_w + 1) / 2 FP32 FMAs;
                HBM  45 B per query (xq 12, sign 1; sdf, var_sdf, var_f, winner, flags 4 each, grad 12) + every
                cell's members once (float4 position/alpha + sigma^2: 20 B) + the winners' FP32 L^-1 triangle;
      adjoint   MUFU  N_w + per touched cell N_c (N_c - 1) (alpha-path kernel entries);
                FP32 lane ops 25 N_w + per touched cell 10 N_c (N_c - 1) + 2 N_c^2 (two FP32 L^-1 products);
                FP64 flops per touched cell 2 N_c^2 (one refinement residual);
                HBM  45 B per query (xq, sign, winner, d_sdf, d_grad, d_xq) + 24 B per sample (d_x read and
                written) + the touched cells' members, FP32 L^-1 and FP64 L triangles."""
    from paper_2603_29227_gb300 import ksdf

    keys, status, off, mem = ksdf.ksdf_get_cells(h)
    nsz = np.diff(off).astype(np.float64)
    qk = np.empty(len(w.xq), np.uint64)
    ksdf.ksdf_bin(h, np.ascontiguousarray(w.xq, dtype=np.float64), len(w.xq), qk)
    ub, inv = np.unique(qk, return_inverse=True)
    K = w.params["k_cand"]
    cand = np.empty((len(ub), K), np.int32)
    cnt = np.empty(len(ub), np.int32)
    ksdf.ksdf_candidates(h, ub, len(ub), cand, cnt)
    per_bin = np.where(cand >= 0, nsz[np.maximum(cand, 0)], 0).sum(axis=1)
    C = float(per_bin[inv].sum())
    wn = np.asarray(winner)
    ok = wn >= 0
    nw = nsz[wn[ok]]
    Q = len(w.xq)
    tc_sel = nw <= 256
    touched = np.unique(wn[ok])
    nc = nsz[touched]
    tri = lambda n: n * (n + 1) / 2  # noqa: E731
    fwd = {"mufu": C + 3 * nw.sum() + 3 * Q,
           "fp32": 8 * C + 18 * nw.sum() + tri(nw[~tc_sel]).sum(),
           "tc": 6 * tri(nw[tc_sel]).sum(),
           "hbm": 45.0 * Q + 20.0 * nsz.sum() + 4.0 * tri(nc).sum(), "fp64": 0.0}
    bwd = {"mufu": nw.sum() + (nc * (nc - 1)).sum(),
           "fp32": 25 * nw.sum() + (10 * nc * (nc - 1) + 2 * nc ** 2).sum(),
           "tc": 0.0,
           "hbm": 45.0 * Q + 24.0 * len(w.x) + (20.0 * nc + 12.0 * tri(nc)).sum(), "fp64": (2 * nc ** 2).sum()}
    stats = {"C_per_query": C / Q, "Nw_mean": float(nw.mean()) if nw.size else 0.0,
             "Nw_max": int(nw.max()) if nw.size else 0, "touched_cells": int(len(touched)), "cells": int(len(nsz))}
    return fwd, bwd, stats, nsz


def roofline_of(work, seconds, peaks):
    """The binding unit of `work` (max over units of count / peak) and the achieved fraction of it in
    `seconds`.  Peaks: units per second."""
    t = {u: work[u] / peaks[u] for u in ("mufu", "fp32", "tc", "hbm", "fp64") if work.get(u) and peaks.get(u)}
    unit = max(t, key=t.get)
    names = {"mufu": ("alu", "Tops/s (MUFU ex2)"), "fp32": ("alu", "Tops/s (FP32 lane ops)"),
             "tc": ("tensor", "TFLOP/s (TF32)"), "hbm": ("hbm", "GB/s"), "fp64": ("alu", "TFLOP/s (FP64)")}
    scale = 1e9 if unit == "hbm" else 1e12
    achieved = work[unit] / seconds / scale
    peak = peaks[unit] / scale
    return {"bound": names[unit][0], "binding_unit": unit, "achieved": achieved, "peak": peak,
            "unit": names[unit][1], "frac": achieved / peak, "roofline_ms": 1e3 * t[unit], "measured_ms": 1e3 * seconds,
            "unit_ms": {u: round(1e3 * v, 4) for u, v in t.items()}}


def source_digest():
    """Digest of the query and adjoint kernel sources: DRAM traffic recorded from ncu applies only to the
    kernels it was captured from."""
    import hashlib

    hs = hashlib.sha256()
    for f in ("ksdf_query.cu", "ksdf_backward.cu", "ksdf_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2603_29227_gb300", "csrc", f), "rb") as fh:
            hs.update(fh.read())
    return hs.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes (read + write) of one query + adjoint from the committed ncu summary, if it was captured
    from the current kernel sources; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    txt = open(TRAFFIC_FILE).read()
    m = re.search(r"^source_digest\s+([0-9a-f]+)\s*$", txt, re.M)
    t = re.search(r"^query_adjoint_dram_bytes\s+([0-9.eE+]+)\s*$", txt, re.M)
    if not m or not t or m.group(1) != source_digest():
        return None
    return float(t.group(1))


# ----------------------------------------------------------------------------------------------------


def _timed(torch, fn, steps, warmup=3):
    """Mean ms of fn() over `steps` runs timed with CUDA events on the current stream (after `warmup`)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def full_step_bench(torch, dev, ksdf, w, steps=10):
    """fit + query + adjoint of a workload, the query and adjoint replayed from a CUDA graph; ms per step."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    x, var, nrm, xq, sign = t(w.x), t(w.var), t(w.normals), t(w.xq), t(w.sign)
    Q = len(w.xq)
    d_sdf = torch.ones(Q, dtype=torch.float32, device=dev)
    d_grad = torch.full((Q, 3), 0.1, dtype=torch.float32, device=dev)
    m = ksdf.KernelSDF(w.params)
    m.fit(x, var, nrm)
    m.autotune()
    m.autotune_query(xq, sign)
    for _ in range(3):
        o = m.query(xq, sign)
        m.backward(xq, o["winner"], d_sdf, d_grad, sign)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        o = m.query(xq, sign)
        m.backward(xq, o["winner"], d_sdf, d_grad, sign)

    def step():
        m.fit(x, var, nrm)
        g.replay()

    ms = _timed(torch, step, steps)
    qb = _timed(torch, g.replay, steps)
    m.sync_status()
    del m, g
    return {"ms_per_step": ms, "queries_per_s": Q / (ms * 1e-3), "query_adjoint_ms": qb, "fit_ms": ms - qb}


def other_configs(torch, dev, ksdf, main_name):
    """The other synthetic workloads, one GPU, device-resident inputs, CUDA-event timing (warm-up 3)."""
    from paper_2603_29227_gb300 import scenes

    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    res = {}
    # the other 3D workload's full step
    other = "room3d" if main_name == "scale3d" else "scale3d"
    w = scenes.workload(other)
    r = full_step_bench(torch, dev, ksdf, w, steps=10 if other == "room3d" else 3)
    r["workload"] = WORKLOAD_TEXT[other]
    res[other + "_full_step"] = r
    # 2D plain FP64: fit + FP64 query of the 128 x 128 grid (latency bound: microseconds)
    w = scenes.workload("plane2d")
    m = ksdf.KernelSDF(w.params)
    x, var, nrm, sg = t(w.x), t(w.var), t(w.normals), t(w.sign)
    xq64 = t(w.xq.astype(np.float64))
    m.fit(x, var, nrm)
    fit_ms = _timed(torch, lambda: m.fit(x, var, nrm), 10)
    q_ms = _timed(torch, lambda: m.query(xq64, sg, f64=True), 10)
    res["plane2d_fp64"] = {"workload": "10x10 m box + 20 circles, 2,000 samples, 1 m cells; 128^2 grid queries; "
                                       "plain FP64 path", "fit_us": 1e3 * fit_ms, "query_us": 1e3 * q_ms,
                           "queries_per_s": len(w.xq) / (q_ms * 1e-3)}
    del m
    # differentiation: 2,097,152 trajectory queries, forward sdf + grad and the adjoint (model fitted once)
    w = scenes.workload("traj3d")
    m = ksdf.KernelSDF(w.params)
    x, var, nrm, xq = t(w.x), t(w.var), t(w.normals), t(w.xq)
    m.fit(x, var, nrm)
    Q = len(w.xq)
    d_sdf = torch.ones(Q, device=dev)
    d_grad = torch.zeros((Q, 3), device=dev)

    def fb():
        o = m.query(xq, None, ksdf.OUT_SDF | ksdf.OUT_GRAD | ksdf.OUT_WINNER | ksdf.OUT_FLAGS)
        m.backward(xq, o["winner"], d_sdf, d_grad)

    ms = _timed(torch, fb, 10)
    res["traj3d_adjoint"] = {"workload": "room scene, 4,096 trajectories x 64 waypoints x 8 spheres = 2,097,152 "
                                         "queries; sdf + grad forward and adjoint to queries and samples",
                             "ms_per_step": ms, "queries_per_s": Q / (ms * 1e-3)}
    del m, d_sdf, d_grad
    # streaming: LiDAR frames of a city block (scans made on the host by a process pool); frame 0 fits, every later
    # frame appends its hits (ksdf_update) and answers 1M queries around the pose; once refitting every changed
    # cell (the model stays a fresh fit of all samples), once with a refit budget per frame (the training queue)
    city = scenes.make_city()
    n_frames = len(city.poses)
    import multiprocessing as mpc

    with mpc.get_context("spawn").Pool(processes=min(16, os.cpu_count() or 1)) as pool:
        scans = pool.map(city.scan, range(n_frames))
    streams = {}
    for mode, budget in (("exact", 0), ("scheduled", CITY_REFIT_BUDGET)):
        m = ksdf.KernelSDF(city.params)
        ksdf.ksdf_set_schedule(m.h, budget, 1e-3)
        rec = {"refit_ms": [], "query_ms": [], "cells_refit": [], "cells": [], "samples": []}
        S = 0
        for f in range(n_frames):
            hx, hv, hn = (t(a) for a in scans[f])
            xq = t(city.queries(f, 1_000_000))
            torch.cuda.synchronize()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            if f == 0:
                m.fit(hx, hv, hn)
                nref = int(ksdf.ksdf_model_size(m.h)[0])
            else:
                nref = m.update(hx, hv, hn)
            e[1].record()
            m.query(xq)
            e[2].record()
            torch.cuda.synchronize()
            S += int(hx.shape[0])
            rec["refit_ms"].append(round(e[0].elapsed_time(e[1]), 3))
            rec["query_ms"].append(round(e[1].elapsed_time(e[2]), 3))
            rec["cells_refit"].append(nref)
            rec["cells"].append(int(ksdf.ksdf_model_size(m.h)[0]))
            rec["samples"].append(S)
        upd = slice(1, None)
        tot = sum(rec["refit_ms"][upd]) + sum(rec["query_ms"][upd])
        rec["queries_per_s_incl_refit"] = 1e6 * (n_frames - 1) / (tot * 1e-3)
        rec["refit_ms_mean"] = float(np.mean(rec["refit_ms"][upd]))
        rec["query_ms_mean"] = float(np.mean(rec["query_ms"][upd]))
        rec["refit_budget"] = budget
        streams[mode] = rec
        del m
    res["city_stream"] = {"workload": "100x100 m city block, %d frames of a 64x2048 LiDAR scan (~125k hits each, range "
                                      "noise 0.02 m) on a closed path, 1M queries per frame in the 40x40x6 m box "
                                      "around the pose; the GP is fed the raw hits (the BHM front-end runs on the same "
                                      "frames in city_frontend)" % n_frames,
                          "exact": streams["exact"], "scheduled": streams["scheduled"]}
    res["city_frontend"] = city_frontend(torch, dev, city, scans)
    return res


def city_pipeline(torch, dev, city, scans, n_frames):
    """The paper's data flow on the first frames of the city stream, with a persistent map: per frame, the BHM
    update and its surface points (with sigma_i^2); the GP buffer update -- the points of re-marched edges are
    replaced by the new march (ksdf_bhm_edges_marked, ksdf_update_replace), every changed cell refitted -- and the
    SDF query of the frame's 1M points signed by the BHM."""
    from paper_2603_29227_gb300 import bhm, ksdf, scenes

    m = bhm.BHMap(scenes.CITY_BHM, max_blocks=200_000, max_marked=100_000)
    gp = ksdf.KernelSDF(dict(city.params, sign_mode=0))
    ms = {"frontend": [], "gp_update": [], "query": []}
    finite, refit, S = [], [], []
    gkeys = None
    for f in range(n_frames):
        hx = torch.from_numpy(scans[f][0]).to(dev)
        xq = torch.from_numpy(city.queries(f, 1_000_000)).to(dev)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        m.update(city.poses[f], hx)
        x, var, _, k = m.march(device=dev)
        sg = m.query(xq, bhm.BHM_SIGN)["sign"]
        e[1].record()
        if gkeys is None:
            gp.fit(x, var, None)
            n = len(x)
            gkeys = k.clone()
        else:
            drop = m.edges_marked(gkeys)
            n = gp.update_replace(drop, x, var)
            gkeys = torch.cat([gkeys[drop == 0], k])
        e[2].record()
        o = gp.query(xq, sg, ksdf.OUT_SDF | ksdf.OUT_GRAD | ksdf.OUT_VAR_SDF | ksdf.OUT_WINNER | ksdf.OUT_FLAGS)
        e[3].record()
        torch.cuda.synchronize()
        ms["frontend"].append(e[0].elapsed_time(e[1]))
        ms["gp_update"].append(e[1].elapsed_time(e[2]))
        ms["query"].append(e[2].elapsed_time(e[3]))
        finite.append(float(torch.isfinite(o["sdf"]).float().mean()))
        refit.append(int(n))
        S.append(int(gp.S))
    m.sync_status()
    # frame 0 fits and frame 1 makes the first update (its one-time costs: first launches, workspace growth); the
    # rates are those of the frames after
    steady = slice(2, None)
    tot = sum(sum(v[steady]) for v in ms.values())
    return {"frames": n_frames, "frames_timed": n_frames - 2, "frames_per_s": (n_frames - 2) / (tot * 1e-3),
            "frontend_ms_mean": float(np.mean(ms["frontend"][steady])),
            "gp_update_ms_mean": float(np.mean(ms["gp_update"][steady])),
            "query_ms_mean": float(np.mean(ms["query"][steady])),
            "first_fit_ms": float(ms["gp_update"][0]), "first_update_ms": float(ms["gp_update"][1]),
            "cells_refit_mean": float(np.mean(refit[steady])), "gp_samples_final": S[-1],
            "finite_sdf_fraction": float(np.mean(finite))}


def city_frontend(torch, dev, city, scans):
    """The BHM front-end (include/ksdf_bhm.h) on every frame of the city stream: the update (samples along the
    rays, two EM rounds, tau, marks), the surface points of the marked cells, and the BHM sign of the frame's 1M
    queries; then the oracle on a bounded sample of one frame."""
    import time

    from paper_2603_29227_gb300 import bhm, scenes

    m = bhm.BHMap(scenes.CITY_BHM, max_blocks=200_000, max_marked=100_000)
    rec = {"update_ms": [], "march_ms": [], "sign_ms": [], "samples": [], "features": [], "points": [], "blocks": []}
    hits_total = 0
    for f in range(len(scans)):
        hx = torch.from_numpy(scans[f][0]).to(dev)
        xq = torch.from_numpy(city.queries(f, 1_000_000)).to(dev)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        m.update(city.poses[f], hx)
        e[1].record()
        pts = m.march(device=dev)
        e[2].record()
        m.query(xq, bhm.BHM_SIGN)
        e[3].record()
        torch.cuda.synchronize()
        nb, ns, nf = m.size(features=True)
        hits_total += int(hx.shape[0])
        rec["update_ms"].append(round(e[0].elapsed_time(e[1]), 3))
        rec["march_ms"].append(round(e[1].elapsed_time(e[2]), 3))
        rec["sign_ms"].append(round(e[2].elapsed_time(e[3]), 3))
        rec["samples"].append(ns)
        rec["features"].append(nf)
        rec["points"].append(int(len(pts[0])))
        rec["blocks"].append(nb)
    m.sync_status()
    F = len(scans)
    tot_ms = sum(rec["update_ms"]) + sum(rec["march_ms"]) + sum(rec["sign_ms"])
    pipeline = city_pipeline(torch, dev, city, scans, 20)
    out = {"workload": "the city stream's %d LiDAR frames through the BHM map (hinge spacing 0.175 m, 8^3 hinges "
                       "per block, l = 0.11 m, free samples every 0.175 m, 2 EM rounds, marching at 0.0875 m); per "
                       "frame: update, surface points, sign of the 1M queries" % F,
           "frames_per_s": F / (tot_ms * 1e-3), "hits_per_s": hits_total / (tot_ms * 1e-3),
           "samples_per_s_update": sum(rec["samples"]) / (sum(rec["update_ms"]) * 1e-3),
           "update_ms_mean": float(np.mean(rec["update_ms"])), "march_ms_mean": float(np.mean(rec["march_ms"])),
           "sign_ms_mean": float(np.mean(rec["sign_ms"])),
           "samples_per_frame": float(np.mean(rec["samples"])),
           "features_per_sample": float(np.sum(rec["features"]) / max(1, np.sum(rec["samples"]))),
           "points_per_frame": float(np.mean(rec["points"])), "blocks_final": rec["blocks"][-1],
           "tau_final": m.tau, "pipeline": pipeline, "per_frame": rec}
    # the oracle on a bounded sample: 1,200 hits of frame 0 within 10 m of the sensor
    try:
        from oracle import bhm as obhm

        p, hits = scenes.city_bhm_frame(city, 0, radius=10.0, max_hits=1200)
        ob = obhm.BHMOracle(obhm.BHMParams(**scenes.CITY_BHM))
        t0 = time.perf_counter()
        ob.update(p, hits)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"kind": "oracle", "cores": 1, "sample": "update of 1,200 hits of frame 0 within 10 m "
                               "(%d samples), binary64 numpy" % ob.last_samples,
                               "value": ob.last_samples / dt, "unit": "samples/s"}
    except Exception as exc:  # the oracle is test infrastructure; its absence must not stop the bench
        out["cpu_baseline"] = {"unavailable": str(exc)[:200]}
    del m
    return out


def parity_block(w, sel, ref, om, got):
    """This run's outputs on the oracle's sample: SDF for every query; where the GPU picked another winner
    than the oracle (a near tie), the other outputs against the oracle evaluated on the GPU's winner;
    gradient angle excluding only medial-axis queries (cancellation ratio < 1e-2) and zero gradients."""
    gw = got["winner"][sel].astype(np.int64)
    rw = ref["winner"].astype(np.int64)
    fin = np.isfinite(ref["sdf"])
    sdf_err = np.abs(got["sdf"][sel].astype(np.float64) - ref["sdf"])
    diff = (gw != rw) & fin & (gw >= 0)
    rg, rvs, rvf = ref["grad"].copy(), ref["var_sdf"].copy(), ref["var_f"].copy()
    if diff.any():
        alt = om.eval_cell(w.xq[sel][diff], gw[diff].astype(np.int32), w.sign[sel][diff])
        rg[diff], rvs[diff], rvf[diff] = alt["grad"], alt["var_sdf"], alt["var_f"]
    tie_flag = (got["flags"][sel].astype(np.int64) & 4) != 0
    # medial-axis exclusion: cancellation ratio of the gradient sum on the GPU's winner (oracle side)
    keys, status, off, mem = om.cells()
    lam = w.params["lambda"]
    ratio = np.ones(len(sel))
    xs_q = w.xq[sel].astype(np.float64)
    for g in np.unique(gw[fin & (gw >= 0)]):
        s = np.nonzero((gw == g) & fin)[0]
        xs = om.x[mem[off[g]:off[g + 1]]]
        al = om.alpha(int(g))
        r = xs_q[s][:, None, :] - xs[None, :, :]
        r2 = np.sum(r * r, axis=2)
        kp = np.exp(-lam * (r2 - r2.min(axis=1, keepdims=True)))
        num = np.linalg.norm(np.sum((al * kp)[:, :, None] * r, axis=1), axis=1)
        den = np.sum(np.abs(al) * kp * np.sqrt(r2), axis=1)
        ratio[s] = num / np.maximum(den, 1e-300)
    gg = got["grad"][sel].astype(np.float64)
    cosang = np.sum(gg * rg, 1) / np.maximum(np.linalg.norm(gg, axis=1) * np.linalg.norm(rg, axis=1), 1e-300)
    ang = np.degrees(np.arccos(np.clip(cosang, -1, 1)))
    zero = ((got["flags"][sel].astype(np.int64) | ref["flags"].astype(np.int64)) & 8) != 0
    gsel = fin & (ratio >= 1e-2) & ~zero
    vs = np.abs(got["var_sdf"][sel] - rvs) / np.maximum(np.abs(rvs), 1e-30)
    vf = np.abs(got["var_f"][sel] - rvf) / np.maximum(rvf, 1e-3)
    return {"sample": int(len(sel)), "sdf_max_err_m": float(sdf_err[fin].max()),
            "sdf_within_1e-4": bool(sdf_err[fin].max() <= 1e-4),
            "winner_agree": float(np.mean(gw[fin] == rw[fin])),
            "winner_disagree_flagged": float(np.mean(tie_flag[diff])) if diff.any() else 1.0,
            "grad_angle_max_deg": float(ang[gsel].max()) if gsel.any() else 0.0,
            "grad_medial_excluded": int(np.sum(fin & (ratio < 1e-2))),
            "var_sdf_max_rel": float(vs[fin].max()), "var_f_max_scaled": float(vf[fin].max()),
            "note": "per-query checks at every size are the GPU tests (tests/test_gpu_full.py)"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2603_29227_gb300 import ksdf, peaks

    ksdf.load()
    w = make_workload(args, rank)
    Q, S = len(w.xq), len(w.x)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    x, var, nrm, xq, sign = t(w.x), t(w.var), t(w.normals), t(w.xq), t(w.sign)
    gen = torch.Generator(device=dev).manual_seed(5 + rank)
    d_sdf = torch.ones(Q, dtype=torch.float32, device=dev)
    d_grad = torch.randn((Q, 3), generator=gen, device=dev, dtype=torch.float32) * 0.1
    model = ksdf.KernelSDF(w.params)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        model.fit(x, var, nrm)
        out = model.query(xq, sign)
        dq, dx = model.backward(xq, out["winner"], d_sdf, d_grad, sign)
        return out, dq, dx

    # the fit's tile shape (warps per cell, by cell size) and the query's tile shapes picked by timing the
    # candidates on this model and batch
    model.fit(x, var, nrm)
    tune_idx, tune_ms = model.autotune()
    qtune_idx, qtune_ms = model.autotune_query(xq, sign)
    for _ in range(max(args.warmup, 3)):
        out, dq, dx = step()
    torch.cuda.synchronize()
    model.sync_status()
    # the query and its adjoint allocate nothing after the warm-up (workspaces sized): capture them once in a
    # CUDA graph and replay it per step after the (eager) fit, which sizes its launches on the host
    graph_launches = 0
    graph = None
    if not args.no_graph:
        _, l0 = ksdf.ksdf_profile_read(model.h)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            out_g = model.query(xq, sign)
            dq_g, dx_g = model.backward(xq, out_g["winner"], d_sdf, d_grad, sign)
        _, l1 = ksdf.ksdf_profile_read(model.h)
        graph_launches = int(l1 - l0)
        eager_step = step

        def step():
            model.fit(x, var, nrm)
            graph.replay()
            return out_g, dq_g, dx_g

        for _ in range(2):
            out, dq, dx = step()
        torch.cuda.synchronize()
        model.sync_status()
    # timed region
    ksdf.ksdf_profile(model.h, 1)
    _, launches0 = ksdf.ksdf_profile_read(model.h)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)  # L2 flush between steps (outside the events)
        ev[i][0].record()
        out, dq, dx = step()
        ev[i][1].record()
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    stages, launches1 = ksdf.ksdf_profile_read(model.h)
    launches1 += graph_launches * args.steps  # kernels replayed from the graph
    ksdf.ksdf_profile(model.h, 0)
    model.sync_status()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    total_s, value = whole_job_rate(float(step_ms.sum()) / 1e3, world, Q, args.steps, dev)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- query + adjoint alone (the graph), L2 flushed before each replay, and per-stage times ----
    qb_ms = None
    if graph is not None:
        e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in e:
            flush.fill_(1)
            a.record()
            graph.replay()
            b.record()
        torch.cuda.synchronize()
        qb_ms = float(np.mean([a.elapsed_time(b) for a, b in e]))
        # per-stage times of the query and the adjoint (inside the graph) from two eager profiled steps
        ksdf.ksdf_profile(model.h, 1)
        ksdf.ksdf_profile_read(model.h)
        for _ in range(2):
            eager_step()
        torch.cuda.synchronize()
        st2, _ = ksdf.ksdf_profile_read(model.h)
        ksdf.ksdf_profile(model.h, 0)
        for k, v in st2.items():
            if k.startswith("query") or k.startswith("backward"):
                stages[k] = v
    per = {k: v[0] / max(v[1], 1) for k, v in stages.items()}
    if qb_ms is None:
        qb_ms = per.get("query", 0.0) + per.get("backward", 0.0)

    # ---- peaks of this GPU (probes, outside the timed region) ----
    pk = peaks.measure_all()
    mp = json.load(open(MEASURED)) if os.path.exists(MEASURED) else {}
    hbm_gbs = mp.get("hbm_gbs")
    peak_src = "MEASURED_PEAKS.json hbm_gbs" if hbm_gbs else "recipe fallback 6800 GB/s"
    hbm_gbs = hbm_gbs or 6800.0
    P = {"mufu": pk.get("mufu_ex2_tops"), "fp32": pk.get("fp32_ffma_tops"), "tc": pk.get("tf32_tcgen05_tflops"),
         "hbm": hbm_gbs * 1e-3, "fp64": pk.get("fp64_dfma_tflops")}
    P = {u: v * 1e12 for u, v in P.items() if v}  # units per second

    # ---- rooflines ----
    win = out["winner"].cpu().numpy()
    fwd, bwd, wstats, nsz = query_work(w, model.h, win)
    both = {u: fwd[u] + bwd[u] for u in fwd}
    roof = roofline_of(both, qb_ms * 1e-3, P)
    roof["kernel"] = "query + adjoint (all their kernels, one CUDA graph)"
    roof["traffic"] = recorded_traffic()
    roof["algorithmic_bytes"] = both["hbm"]
    roof["peak_source"] = ("probes of libksdf_peaks.so on this GPU (MUFU ex2, FP32 FFMA lane ops, tcgen05 TF32, "
                           "FP64 DFMA), measured live; HBM: " + peak_src + " (of measured)")
    rooflines = {"query": roofline_of(fwd, per.get("query", qb_ms) * 1e-3, P),
                 "adjoint": roofline_of(bwd, per.get("backward", qb_ms) * 1e-3, P)}
    if "fit.cholesky" in per and "fp64" in P:
        fl64 = fit_fp64_flops(nsz)
        rooflines["fit.cholesky"] = {"bound": "alu", "unit": "TFLOP/s (FP64)",
                                     "achieved": fl64 / (per["fit.cholesky"] * 1e-3) / 1e12, "peak": P["fp64"] / 1e12,
                                     "nominal_peak": 1.25,
                                     "what": "FP64 flops of the factorisation: N^3/3 + 2 N^2 per cell, over the "
                                             "factorisation stage, which also runs most of the FP32 L^-1 kernels "
                                             "(high-priority streams beside the FP64 classes)",
                                     "stage_ms": per["fit.cholesky"], "linv_tail_ms": per.get("fit.linv")}
        rooflines["fit.cholesky"]["frac"] = rooflines["fit.cholesky"]["achieved"] / rooflines["fit.cholesky"]["peak"]

    # ---- plain FP64 query on the same inputs (outside the timed region) ----
    xq64 = xq.double()
    model.query(xq64, sign, f64=True)
    torch.cuda.synchronize()
    ksdf.ksdf_profile(model.h, 1)
    model.query(xq64, sign, f64=True)
    st64, _ = ksdf.ksdf_profile_read(model.h)
    ksdf.ksdf_profile(model.h, 0)
    del xq64
    q64_ms = st64["query64"][0] / st64["query64"][1]
    q32_ms = per.get("query", float("nan"))

    # ---- end to end through the C ABI with pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        hx, hv, hn, hq, hs = pin(w.x), pin(w.var), pin(w.normals), pin(w.xq), pin(w.sign)
        hds, hdg = d_sdf.cpu().pin_memory(), d_grad.cpu().pin_memory()
        outs = [torch.empty(Q, dtype=torch.float32).pin_memory(), torch.empty((Q, 3), dtype=torch.float32).pin_memory(),
                torch.empty(Q, dtype=torch.float32).pin_memory(), torch.empty(Q, dtype=torch.float32).pin_memory(),
                torch.empty(Q, dtype=torch.int32).pin_memory(), torch.empty(Q, dtype=torch.int32).pin_memory()]
        hdq = torch.empty((Q, 3), dtype=torch.float32).pin_memory()
        hdx = torch.zeros((S, 3), dtype=torch.float32).pin_memory()
        h = model.h
        ksdf.ksdf_set_stream(h, torch.cuda.current_stream().cuda_stream)

        def e2e_step():
            ksdf.ksdf_fit(h, hx, hv, hn, S)
            ksdf.ksdf_query(h, hq, Q, hs, ksdf.OUT_ALL, *outs)
            ksdf.ksdf_query_backward(h, hq, Q, hs, outs[4], hds, hdg, hdq, hdx)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(3, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h2d = sum(a.numel() * a.element_size() for a in (hx, hv, hn, hq, hs)) + \
            sum(a.numel() * a.element_size() for a in (hq, hs, outs[4], hds, hdg, hdx))
        d2h = sum(a.numel() * a.element_size() for a in outs) + hdq.numel() * 4 + hdx.numel() * 4
        e2e = {"value": Q * n_e2e / (t1 - t0), "unit": "queries/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
               "how": "ksdf_fit/ksdf_query/ksdf_query_backward with pinned host arrays; the library copies "
                      "in and out inside each call; host wall clock"}
        del hx, hv, hn, hq, hs, hds, hdg, outs, hdq, hdx

    # ---- CPU FP64 oracle: baseline timing and the parity of this run's outputs on its sample ----
    cpu = None
    parity = None
    if not args.no_cpu:
        import oracle

        oracle.build()
        threads = oracle.set_threads(os.cpu_count() or 1)
        sel, cd_sdf, cd_grad = oracle_sample(w, args.cpu_sample)
        fit_s, qb_s = [], []
        for _ in range(max(1, args.cpu_repeats)):
            tf, tq, ref, om = oracle_step(w, sel, cd_sdf, cd_grad)
            fit_s.append(tf)
            qb_s.append(tq)
        cpu = oracle_stats(w, sel, fit_s, qb_s, threads)
        got = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        parity = parity_block(w, sel, ref, om, got)
        del om

    cfg = workload_config(w, args)  # the same block as the reference arm's
    run = {"cells": int(len(nsz)), "work": wstats,
                "launch": ("fit launched from the host (it sizes its launches on the host); query + adjoint replayed "
                           "from one CUDA graph captured after the warm-up" if not args.no_graph
                           else "all launched from the host"),
                "fit_autotune": {"table": tune_idx, "fit_ms_per_table": [round(float(v), 3) for v in tune_ms]},
                "query_autotune": {"choice": qtune_idx, "query_ms_per_pair": [round(float(v), 3) for v in qtune_ms],
                                   "pairs": "3 x phase A budget (64, 128, 256 chunks) + phase B class split (64, "
                                            "96, 128 samples)"},
                "precision": "FP64 kernel matrix (entries above 2.4e-16; smaller ones in FP32), Cholesky and alpha; "
                             "FP32 L^-1; FP32 query with compensated mean; V[f] contraction on tcgen05 in TF32 split "
                             "three ways with FP32 accumulation; FP32 adjoint with one FP64 refinement of each cell "
                             "solve"}
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(step_ms.mean()), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic", "config": cfg,
        "run": run,
        "roofline": roof,
        "rooflines": rooflines,
        "peaks_measured": pk,
        "stage_ms": {k: round(v, 4) for k, v in per.items()},
        "query_adjoint_ms": qb_ms,
        "plain_fp64": {"query_ms": q64_ms, "mixed_query_ms": q32_ms, "query_speedup": q64_ms / q32_ms},
        "cpu_baseline": cpu,
        "parity": parity,
        "e2e": e2e,
        "gpu_launches": int(launches1 - launches0),
        "clocks": clk,
        "wall_s": wall1 - wall0,
        "step_ms_min_median_max": [float(step_ms.min()), float(np.median(step_ms)), float(step_ms.max())],
    }
    if not args.no_others and world == 1:
        # the optional SDF-gradient variance on this workload: the same forward with and without it
        base_ms = _timed(torch, lambda: model.query(xq, sign), 3)
        vg_ms = _timed(torch, lambda: model.query(xq, sign, mask=ksdf.OUT_ALL | ksdf.OUT_VAR_GRAD), 3)
        vg = {"workload": w.name + ": forward with the SDF-gradient variance output (Sec. IV-B.3, App. C)",
              "query_ms": base_ms, "query_with_var_grad_ms": vg_ms, "var_grad_extra_ms": vg_ms - base_ms,
              "queries_per_s_with_var_grad": Q / (vg_ms * 1e-3)}
        del model, graph
        torch.cuda.empty_cache()
        line["other_configs"] = other_configs(torch, dev, ksdf, w.name)
        line["other_configs"][w.name + "_var_grad"] = vg
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

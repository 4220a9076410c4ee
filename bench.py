#!/usr/bin/env python
"""Throughput of the FKP power-spectrum multipole path on GB300.

Workload (one step = one mock): the BOSS-like survey -- L = 3500 Mpc/h box,
512^3 grid, TSC assignment, observer at the box centre, 10,000 deg^2 cap,
1100 < r < 1700 Mpc/h, Gaussian nbar(r) peaking at 4e-4, ~7.0e5 lognormal
galaxies with radial RSD (f = 0.7) and 3.5e7 randoms (50x), FKP P0 = 1e4;
P_0, P_2, P_4 (22 moment fields) and P_4b in 60 bins of 0.005 h/Mpc.
Each step runs scalars, gridding, the three FFT passes with moment fields,
grouping, Legendre recombination and binning, and copies P_l to the host.
Inputs (0.57 GB catalog, 1.07 GB grid, 17 GB of FFT intermediates) are all
larger than L2, so no L2 flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 oracle on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "mocks/s for P_l=0,2,4 (512^3) and B_l (k<=0.2), served vs plain; p99 latency"
WORKLOAD = "BOSS-like P_0,2,4 + P_4b: L=3500 Mpc/h, 512^3 TSC, 7.0e5 galaxies + 3.5e7 randoms, 60 bins dk=0.005"
BINS = (0.0, 0.005, 60)
BALL = 1 | 2 | 4 | 8 | 16 | 32 | 64  # P_0,2,4, P_4b, B_0,2,4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-slots", type=int, default=2, help="server slots for the end-to-end leg (1: plain calls)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-cores", type=int, default=0, help="reference arm: cores the oracle may use (0: all)")
    ap.add_argument("--reference-budget", type=float, default=200.0,
                    help="reference arm: seconds of whole-mock oracle runs (at least one mock runs)")
    ap.add_argument("--cufft", type=int, default=1, help="time cuFFT (torch.fft) as a baseline (0 skips)")
    ap.add_argument("--experiment", default="", choices=["", "p4b", "qell"],
                    help="run a synthetic version of one of the paper's experiments instead of the benchmark")
    ap.add_argument("--experiment-mocks", type=int, default=64)
    ap.add_argument("--experiment-workers", type=int, default=8)
    ap.add_argument("--cached-steps", type=int, default=10,
                    help="timed mocks with the randoms cached on the plan (0 skips that leg)")
    ap.add_argument("--grid", type=int, default=512, help="grid side (512 is the benchmark workload)")
    ap.add_argument("--ran-ratio", type=float, default=50.0, help="randoms per galaxy (50 in the workload)")
    ap.add_argument("--bisp-steps", type=int, default=3, help="timed bispectrum mocks (0 skips the B leg)")
    ap.add_argument("--bisp-grid", type=int, default=360, help="bispectrum grid (360 is the workload)")
    ap.add_argument("--bisp-nshells", type=int, default=37, help="bispectrum shells (37 reach k = 0.2)")
    ap.add_argument("--serve-requests", type=int, default=64, help="requests in the serving leg (0 skips it)")
    ap.add_argument("--serve-plain-requests", type=int, default=32,
                    help="the first this many requests also run through the plain sequential path")
    ap.add_argument("--serve-rate", type=float, default=4.0, help="Poisson arrival rate of the serving leg (req/s)")
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--small-steps", type=int, default=200, help="timed 64^3 mocks per mode (0 skips that leg)")
    ap.add_argument("--batch-mocks", type=int, default=32, help="mocks in the batched leg (0 skips it)")
    ap.add_argument("--batch-oracle-mocks", type=int, default=0,
                    help="batched-leg mocks also compared with the FP64 oracle (tens of seconds each)")
    ap.add_argument("--fused-mocks", type=int, default=64,
                    help="64^3 mocks per fused call in the fused leg (0 skips it; 256^3: a quarter)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# Replicas: mocks are independent, so N GPUs run N replicas, each on its own
# seed, with no collective on the data path; only the timing is combined.

def replica_seed(seed, rank):
    """Each rank's mock seed (the seed range is partitioned by rank)."""
    return seed + rank


def max_over_ranks(x, world):
    """The largest of each rank's x (a time), over the process group."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, seconds_per_mock_max):
    """Whole-job mocks/s: every rank finished one mock per step, the step
    lasting as long as the slowest rank's."""
    return world / seconds_per_mock_max


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"fkp_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes of one mock of the power step: the least traffic the
# method needs (catalog read once, the real grid F written once and read
# once, the k_z-power groups that carry the moment fields through the
# z-FFT written once and read once; half = one half-spectrum field of
# N^2 (N/2 + 1) complex FP32 values), split by stage.  The design's own
# extra traffic (the fixed-point grid is 8 bytes per node, the x-pass spills
# every moment half spectrum for the y-pass to read) is not algorithmic: it
# shows in the measured DRAM `traffic` instead.
# ---------------------------------------------------------------------------

def algorithmic_bytes(N, ngroups, n_obj, cat_bytes=16):
    half = N * N * (N // 2 + 1) * 8
    grid = 4 * N ** 3
    return {
        "count": 0,                                  # reads the catalog, but the step reads it once: counted below
        "assign": cat_bytes * n_obj + grid,          # catalog (x, y, z, nbar) read once; F written once
        "xpass": grid,                               # F read once
        "ypass": ngroups * half,                     # the k_z-power groups written once
        "zpass": ngroups * half,                     # the groups read once (bins are negligible)
    }


PASS_SOURCES = {"xpass": "k_xpass.cu", "ypass": "k_ypass.cu", "zpass": "k_zpass.cu"}


def source_sha(kernel):
    """First 12 hex of sha1 of a pass's sources (its .cu file and the shared
    headers k_fftpass.cuh, fkp_fft.cuh, fkp_kernels.cuh) with comments and
    blank lines removed, so that only code changes disown a recorded capture."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in (PASS_SOURCES[kernel], "k_fftpass.cuh", "fkp_fft.cuh", "fkp_kernels.cuh"):
        src = open(os.path.join(ROOT, "paper_1506_02729_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = [re.sub(r"//.*", "", ln).rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:12]


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or None
    when the kernel's sources changed since the counters were taken."""
    try:
        if kernel not in PASS_SOURCES:
            return None
        sha = source_sha(kernel)
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            if line.startswith("#") or not line.strip():
                continue
            kv = dict(t.split("=", 1) for t in line.split())
            if kv.get("kernel") == kernel and kv.get("src_sha1") == sha:
                return int(kv["bytes"])
    except Exception:
        return None
    return None


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# oracle baseline on a bounded sample
# ---------------------------------------------------------------------------

def oracle_full(gal, ran, sv):
    """Wall time of the FP64 oracle (oracle.power.power, as it stands) on one
    whole mock of the workload: scalars, gridding of every galaxy and random,
    the 22 moment-field FFTs, recombination and binning; and its result."""
    from oracle import power as op
    t0 = time.perf_counter()
    ref = op.power(gal, ran, sv.geometry(), BINS)
    return time.perf_counter() - t0, ref


def fp64_errors(got, ref):
    """Largest error of each output of the GPU path against the FP64 oracle on
    the same catalogs: P_l per bin with modes relative to max(|P_l|, |P_0|,
    the raw monopole) (P_2, P_4 and the shot-noise-subtracted P_0 cross zero),
    the scalars relative to themselves, and whether the mode counts agree."""
    m = np.asarray(ref["nmodes"]) > 0
    den = np.maximum(np.abs(ref["P0"][m]), np.abs(ref["mono_raw"][m]))
    out = {}
    for k in ("P0", "P2", "P4", "P4b"):
        d = np.maximum(np.abs(ref[k][m]), den)
        out[k] = float(np.max(np.abs(np.asarray(got[k])[m] - ref[k][m]) / d))
    for k in ("alpha", "I22", "N0"):
        out[k] = float(abs(got[k] / ref[k] - 1.0))
    out["nmodes_equal"] = bool(np.array_equal(np.asarray(got["nmodes"]), np.asarray(ref["nmodes"])))
    return out


def restrict_cores(n):
    """Confines this process (and the FFT worker threads it starts) to its
    first n allowed cores; returns the cores it may now use."""
    try:
        allowed = sorted(os.sched_getaffinity(0))
        if n and n < len(allowed):
            os.sched_setaffinity(0, set(allowed[:n]))
    except Exception:
        pass
    return cores_used()


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------

def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on whole mocks of
    the benchmark workload (one step = one whole mock; no sampling and no
    extrapolation).  A whole mock takes about a minute, so the arm runs as
    many of the requested steps as fit in --reference-budget seconds (at
    least one); the line reports the steps it ran.  Warm-up: one oracle run
    on the small 64^3 survey (imports, page faults), not a workload step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import mockgen
    from oracle import power as op
    cores = restrict_cores(args.oracle_cores)
    small = mockgen.survey_small()
    sg, sr = mockgen.catalog(small, args.seed)
    kf = 2 * math.pi / small.L
    op.power(sg, sr, small.geometry(), (0.5 * kf, kf, 32))
    sv = mockgen.survey_boss()
    gal, ran = mockgen.catalog(sv, args.seed)
    ts = []
    t_start = time.perf_counter()
    while len(ts) < max(1, args.steps):
        ts.append(oracle_full(gal, ran, sv)[0])
        if time.perf_counter() - t_start + ts[-1] > args.reference_budget:
            break
    t_mock = float(np.mean(ts))
    value = 1.0 / t_mock
    desc = (f"oracle (numpy/scipy FP64) on {len(ts)} whole mock(s) of the workload, {cores} core(s), "
            f"{int(gal['x'].size)} galaxies + {int(ran['x'].size)} randoms at 512^3; per mock "
            + ", ".join(f"{t:.1f} s" for t in ts))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "mocks/s", "n_gpus": 1,
            "steps": len(ts), "requested_steps": args.steps, "warmup": 0, "ms_per_step": 1000 * t_mock,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic lognormal mocks (mockgen), seeded per rank",
            "config": workload_config(sv, gal, ran, 1),
            "cpu_baseline": {"value": value, "unit": "mocks/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "mocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(sv, gal, ran, world):
    workload = WORKLOAD if (sv.N == 512 and sv.random_ratio == 50.0) else \
        f"reduced case: {sv.N}^3, randoms x{sv.random_ratio:g} (not the benchmark workload)"
    return {"workload": workload, "grid": sv.N, "n_gal": int(gal["x"].size), "n_ran": int(ran["x"].size),
            "l2": "inputs larger than L2 (no flush needed)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_gpu(args):
    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    from paper_1506_02729_gb300 import build as fbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    fbuild.build()
    sv = mockgen.survey_boss(N=args.grid, random_ratio=args.ran_ratio)
    gal, ran = mockgen.catalog(sv, replica_seed(args.seed, rank))
    n_obj = gal["x"].size + ran["x"].size
    dg = {k: torch.from_numpy(v).cuda() for k, v in gal.items()}
    dr = {k: torch.from_numpy(v).cuda() for k, v in ran.items()}
    geom = sv.geometry()
    plan = fkp.Plan(geom, BINS, device=local)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        plan.power(dg, dr, stream=stream)
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage = []
    e0.record(stream)
    for _ in range(args.steps):
        r = plan.power(dg, dr, stream=stream)
        stage.append(r["timing_ms"].copy())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_all = max_over_ranks(ms, world)
    value = job_rate(world, ms_all / 1000.0)

    # end to end through the C ABI with host (pinned) catalogs
    hg = {k: torch.from_numpy(v).pin_memory() for k, v in gal.items()}
    hr = {k: torch.from_numpy(v).pin_memory() for k, v in ran.items()}
    plan.power(hg, hr, stream=stream)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.power(hg, hr, stream=stream)
    torch.cuda.synchronize()
    sync_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world)
    # the same through the request server (C ABI submit/wait): two slots, so
    # one request's host-to-device copies overlap the other's kernels; every
    # request copies its catalogs in and its bins out
    e2e_s = sync_s
    if args.e2e_slots > 1:
        srv = fkp.Server(nslots=args.e2e_slots, device=local)
        for t in [srv.submit(geom, BINS, hg, hr) for _ in range(args.e2e_slots)]:
            srv.wait(t)
        barrier()
        t0 = time.perf_counter()
        for t in [srv.submit(geom, BINS, hg, hr) for _ in range(args.e2e_steps)]:
            srv.wait(t)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, world)
        srv.close()
    h2d = 16 * n_obj
    d2h = 8 * (6 * 60 + 60) + 8 * 24

    # roofline of the dominant kernel (stage times from CUDA events recorded on
    # the launching stream between the stages of every timed step)
    st = np.mean(np.array(stage), axis=0)
    names = {"count": st[0], "assign": st[1], "xpass": st[2], "ypass": st[3], "zpass": st[4]}
    ab = algorithmic_bytes(sv.N, 9, n_obj)  # 9 k_z-power groups carry P_0,2,4 (and P_4b)
    dom = max(names, key=names.get)
    pk, src = peaks()
    achieved = ab[dom] / (names[dom] * 1e-3) / 1e9
    step_bytes = sum(ab.values())
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": recorded_traffic(dom) if sv.N == 512 else None,
            "algorithmic_bytes": ab[dom], "peak_source": src,
            "stage_ms": {k: float(v) for k, v in names.items()},
            "stage_algorithmic_bytes": ab,
            "stage_frac": {k: ab[k] / (names[k] * 1e-3) / 1e9 / pk["hbm_gbs"] for k in names},
            "step": {"algorithmic_bytes": step_bytes, "ms": ms_all,
                     "frac": step_bytes / (ms_all * 1e-3) / 1e9 / pk["hbm_gbs"]}}

    line = {"metric": METRIC, "value": value, "unit": "mocks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic lognormal mocks (mockgen), seeded per rank",
            "config": workload_config(sv, gal, ran, world),
            "e2e": {"value": job_rate(world, e2e_s), "unit": "mocks/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "path": f"fkp_server_submit/wait, {args.e2e_slots} slots"
                    if args.e2e_slots > 1 else "fkp_power, one call at a time",
                    "one_call_at_a_time": job_rate(world, sync_s)},
            # per step: 2 counts, scalars, tile totals, scan, 2 scatters, L^ab, tiles, x, y, z, bins
            "gpu_launches": 13 * args.steps,
            "roofline": roof,
            "fft_schedule": plan.schedule(),
            "clocks": ck}
    if args.cached_steps > 0:
        line["cached_randoms"] = run_cached(args, plan, dg, dr, r, stream)
    if args.cufft and world == 1 and sv.N == 512:
        line["cufft_baseline"] = run_cufft(args, float(names["xpass"] + names["ypass"] + names["zpass"]))
    if args.small_steps > 0:
        line["small_grid"] = run_small(args, stream)
    if args.bisp_steps > 0:
        line["bispectrum"] = run_bisp(args, gal, ran, dg, dr, stream)
    if args.serve_requests > 0 and world == 1:
        del dg, dr
        torch.cuda.empty_cache()
        line["serving"] = run_serve(args, gal, ran)
    if args.batch_mocks > 0 and world == 1:
        torch.cuda.empty_cache()
        line["batch"] = run_batch(args)
    if args.fused_mocks > 0 and world == 1:
        torch.cuda.empty_cache()
        line["fused"] = run_fused(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_mock, ref = oracle_full(gal, ran, sv)
        line["cpu_baseline"] = {"value": 1.0 / t_mock, "unit": "mocks/s", "cores": cores_used(), "kind": "oracle",
                                "sample": f"oracle (numpy/scipy FP64) on one whole mock of the workload (the "
                                          f"timed catalogs, {sv.N}^3): {t_mock:.1f} s"}
        # the last timed step's outputs against that oracle run
        try:
            line["error_vs_fp64"] = fp64_errors(r, ref)
        except Exception as e:  # the line is printed whatever happens here
            line["error_vs_fp64"] = {"unavailable": f"{type(e).__name__}: {e}"[:120]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_cached(args, plan, dg, dr, ref, stream):
    """Mocks that share one random catalog (the covariance setup of Sec.
    III.C): the randoms are gridded once onto the plan without alpha
    (fkp_plan_cache_randoms) and each step grids only the galaxies and forms
    F = G - alpha R.  Same catalogs as the headline, which grids the randoms
    every step.  Reports mocks/s, the per-stage times and the largest P_l
    difference from the headline path (graded by the raw monopole)."""
    import torch
    t0 = time.perf_counter()
    plan.cache_randoms(dr, stream=stream)
    t_cache = time.perf_counter() - t0
    for _ in range(2):
        plan.power(dg, None, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st = []
    e0.record(stream)
    for _ in range(args.cached_steps):
        r = plan.power(dg, None, stream=stream)
        st.append(r["timing_ms"].copy())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.cached_steps
    m = np.mean(np.array(st), axis=0)
    plan.cache_randoms({k: v[:0] for k, v in dr.items()}, stream=stream)
    return {"what": "randoms gridded once per (footprint, grid); each step grids the galaxies only",
            "value": 1000.0 / ms, "unit": "mocks/s", "ms_per_step": ms, "steps": args.cached_steps,
            "cache_build_s": t_cache,
            "stage_ms": {"count": float(m[0]), "assign_and_combine": float(m[1]), "xpass": float(m[2]),
                         "ypass": float(m[3]), "zpass": float(m[4])},
            "max_rel_diff_vs_headline_P": _rel_diff(r, ref, ("P0", "P2", "P4", "P4b"), np.abs(ref["mono_raw"]))}


def run_cufft(args, pass_ms, N=512, nfields=16):
    """cuFFT (through torch.fft) timed as a baseline beside the hand-written
    passes: one batched 3-D real-to-complex transform of 16 FP32 fields of
    512^3 (the trace-reduced moment fields of one mock), CUDA events on the
    current stream, 3 timed calls after 2 warm-ups.  cuFFT transforms the 16
    fields and stops; the hand-written x, y and z passes also build the
    moment fields, group them by k_z power, recombine the Legendre fields and
    bin them (pass_ms)."""
    import torch
    half = N * N * (N // 2 + 1) * 8
    x = torch.randn(nfields, N, N, N, device="cuda", dtype=torch.float32)
    y = None
    for _ in range(2):
        y = torch.fft.rfftn(x, dim=(-3, -2, -1))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        y = torch.fft.rfftn(x, dim=(-3, -2, -1))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del x, y
    torch.cuda.empty_cache()
    pk, src = peaks()
    moved = nfields * (4 * N ** 3 + half)
    return {"what": f"{nfields} batched 3-D r2c FFTs of {N}^3 FP32 fields (torch.fft.rfftn -> cuFFT)",
            "ms": ms, "io_bytes": moved, "io_frac_of_hbm": moved / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
            "hand_written_passes_ms": pass_ms,
            "note": "the hand-written passes also build the moment fields, group them by k_z power "
                    "(9 groups through the z-FFT), recombine and bin"}


BSHELLS = (3, 3, 3, 37)  # centres 3(s+1) k_f, width 3 k_f, to k = 0.2 h/Mpc


def run_small(args, stream):
    """The small survey (L = 1000 Mpc/h, 64^3 CIC, 2e4 galaxies + 2e5 randoms,
    P_0,2,4 + P_4b in 32 bins): launch-bound, so it is where CUDA-graph replay
    of the power path shows; mocks/s with the graph and with plain launches
    (each call synchronizes and finishes the bins on the host)."""
    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    sv = mockgen.survey_small()
    gal, ran = mockgen.catalog(sv, args.seed)
    dg = {k: torch.from_numpy(v).cuda() for k, v in gal.items()}
    dr = {k: torch.from_numpy(v).cuda() for k, v in ran.items()}
    kf = 2 * np.pi / sv.L
    plan = fkp.Plan(sv.geometry(), (0.5 * kf, kf, 32))
    out = {"workload": "small survey: L=1000 Mpc/h, 64^3 CIC, 2e4 galaxies + 2e5 randoms, 32 bins", "unit": "mocks/s"}
    for name, on in (("graph", True), ("plain", False)):
        plan.set_graphs(on)
        for _ in range(3):
            plan.power(dg, dr, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.small_steps):
            p = plan.power(dg, dr, stream=stream)
        dt = time.perf_counter() - t0
        assert p["graph"] == (1 if on else 0)
        out[name] = {"value": args.small_steps / dt, "ms_per_step": 1000.0 * dt / args.small_steps}
    plan.close()
    return out


def run_bisp(args, gal, ran, dg, dr, stream):
    """B_0,2,4 of the same catalog on a 360^3 TSC grid (37 shells to k = 0.2):
    mocks/s of the whole P + B path and its stage times (CUDA events), for the
    FP32 CUDA-core contraction and the two tcgen05 tensor-core contractions."""
    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    sv = mockgen.survey_boss(N=args.bisp_grid)
    bshells = BSHELLS[:3] + (args.bisp_nshells,)
    plan = fkp.Plan(sv.geometry(), BINS, bshells=bshells, want=127)
    modes = {"fp32": fkp.FKP_CONTRACT_FP32, "bf16x3_tcgen05": fkp.FKP_CONTRACT_BF16X3,
             "bf16x6_tcgen05": fkp.FKP_CONTRACT_BF16X6}
    wl = "B_0,2,4 + P_l: BOSS-like catalog, 360^3 TSC, 37 shells of 3 k_f to k=0.2"
    if (args.bisp_grid, args.bisp_nshells) != (360, 37):
        wl = f"reduced case: {args.bisp_grid}^3, {args.bisp_nshells} shells (not the workload)"
    out = {"workload": wl,
           "ntriangles": int(plan.ntri), "unit": "mocks/s", "modes": {}}
    for name, mode in modes.items():
        plan.bispectrum(dg, dr, contraction=mode, stream=stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st = []
        e0.record(stream)
        for _ in range(args.bisp_steps):
            p, b = plan.bispectrum(dg, dr, contraction=mode, stream=stream)
            st.append(p["timing_ms"].copy())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.bisp_steps
        m = np.mean(np.array(st), axis=0)
        out["modes"][name] = {"value": 1000.0 / ms, "ms_per_step": ms,
                              "stage_ms": {"grids": float(m[0] + m[1]), "F_passes": float(m[2] + m[3] + m[4]),
                                           "Fw_passes_and_shell_ifft": float(m[5]), "contraction": float(m[6])}}
    # the headline is the accurate tensor-core mode (3-way split, within the
    # 1e-4 bar like the FP32 contraction); the hi/lo split is the fast mode,
    # with a random per-product error of ~2^-18
    out["value"], out["mode"] = out["modes"]["bf16x6_tcgen05"]["value"], "bf16x6_tcgen05"
    # rooflines (the survey's accounting for this workload): the contraction's
    # useful tensor work, 2 x (triangles x 3 multipoles) x N^3 multiply-adds
    # times the BF16 products per term (3 hi/lo, 6 for the 3-way split),
    # against the sustained BF16 peak; the rest of the step's algorithmic bytes
    # (catalog 20 B per object, the F and F^w grids written and read, the k_z
    # groups of both pass sets written and read, the 3 S shell fields of both
    # the fields' shell IFFTs written and read) against HBM
    pk, src = peaks()
    N = args.bisp_grid
    N3 = float(N) ** 3
    nout = 3 * int(plan.ntri)
    roof = {}
    for name, nprod in (("bf16x3_tcgen05", 3), ("bf16x6_tcgen05", 6)):
        cms = out["modes"][name]["stage_ms"]["contraction"]
        fl = 2.0 * nout * N3 * nprod
        ach = fl / (cms * 1e-3) / 1e12
        roof[name] = {"bound": "tensor", "kernel": "contraction", "useful_flop": fl, "achieved": ach,
                      "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                      "frac": ach / pk["bf16_tflops_sustained"], "peak_source": src}
    half = N * N * (N // 2 + 1) * 8.0
    nmax = int(3 * args.bisp_nshells + 1.5)
    nobj = int(len(gal["x"]) + len(ran["x"]))
    bts = (20.0 * nobj + 2 * 2 * 4 * N3 + 2 * (2 * 9 * half)
           + 2 * 3 * args.bisp_nshells * ((nmax + 1) * N * N * 8.0))
    st = out["modes"]["bf16x6_tcgen05"]["stage_ms"]
    oms = st["grids"] + st["F_passes"] + st["Fw_passes_and_shell_ifft"]
    roof["grids_passes_shell_ifft"] = {"bound": "hbm", "algorithmic_bytes": bts, "ms": oms,
                                       "achieved": bts / (oms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                       "frac": bts / (oms * 1e-3) / 1e9 / pk["hbm_gbs"], "peak_source": src}
    out["roofline"] = roof
    out["accuracy"] = {"fp32": "within 1e-4 of the FP64 oracle", "bf16x6_tcgen05": "within 1e-4 of the FP64 oracle",
                       "bf16x3_tcgen05": "random per-product error ~2^-18 (triangle sums within 6 x 2^-17 "
                                         "sqrt(sum_x t^2) of the 3-way split)"}
    plan.close()
    return out


def _fused_vs_single(plan, mocks, reps):
    """mocks/s of plan.power_batch over all mocks against one plan.power call
    per mock (device catalogs), and their largest P_l difference."""
    import torch
    gals, rans = [m[0] for m in mocks], [m[1] for m in mocks]
    plan.power_batch(gals, rans)  # the batch workspace
    for g, r in mocks:
        plan.power(g, r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fused = plan.power_batch(gals, rans)
    tf = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        single = [plan.power(g, r) for g, r in mocks]
    ts = (time.perf_counter() - t0) / reps
    diff = max(_rel_diff(a, b, ("P0", "P2", "P4"), np.abs(b["mono_raw"])) for a, b in zip(fused, single))
    st = fused[0]["timing_ms"]
    plan.close()
    return {"mocks": len(mocks), "fused_mocks_per_s": len(mocks) / tf, "single_mocks_per_s": len(mocks) / ts,
            "fused_stage_ms": {"gridding_all": float(st[1]), "xpass": float(st[2]), "ypass": float(st[3]),
                               "zpass_and_bins": float(st[4]), "total": float(st[7])},
            "fused_vs_single_max_rel_diff_P": diff}


def run_fused(args):
    """Several mocks per call (fkp_power_batch: each mock gridded with launches
    shaped by its own catalogs, then one launch per FFT pass and one bin
    reduction for all of them) against one fkp_power call per mock, on two
    ensembles of uneven mocks: the small survey (64^3 CIC; each mock a random
    50-100 % subsample of 2e4 galaxies and of 2e5 randoms), where launches and
    the per-call synchronisation dominate, and BOSS-like mocks on a 256^3 grid
    (N_g uniform in [5e5, 1.2e6], a random subsample of a 1.2e6-galaxy master
    catalog, and 30 N_g randoms).  Device catalogs on both paths; P_0,2,4."""
    import dataclasses

    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    g = np.random.default_rng(args.seed + 700)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed + 701)

    def subsample(cat, n_keep):
        idx = torch.sort(torch.randperm(cat["x"].numel(), device="cuda", generator=gen)[:n_keep]).values
        return {k: v[idx].contiguous() for k, v in cat.items()}

    want = fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4
    out = {"unit": "mocks/s", "path": "fkp_power_batch vs fkp_power per mock"}
    sv = mockgen.survey_small()
    gal, ran = mockgen.catalog(sv, args.seed + 702)
    dg = {k: torch.from_numpy(v).cuda() for k, v in gal.items()}
    dr = {k: torch.from_numpy(v).cuda() for k, v in ran.items()}
    ms = [(subsample(dg, int(g.uniform(0.5, 1.0) * gal["x"].size)), subsample(dr, int(g.uniform(0.5, 1.0) *
                                                                                        ran["x"].size)))
          for _ in range(args.fused_mocks)]
    kf = 2 * np.pi / sv.L
    out["small"] = dict(workload=f"{len(ms)} small-survey mocks, 64^3 CIC, 1e4-2e4 galaxies + 1e5-2e5 randoms",
                        **_fused_vs_single(fkp.Plan(sv.geometry(), (0.5 * kf, kf, 32), want=want), ms, 5))
    del ms, dg, dr
    base = mockgen.survey_boss(N=256)
    svb = dataclasses.replace(base, nbar_peak=base.nbar_peak * 1.2e6 / 7.0e5, random_ratio=30.0)
    gal, ran = mockgen.catalog(svb, args.seed + 703)
    dg = {k: torch.from_numpy(v).cuda() for k, v in gal.items()}
    dr = {k: torch.from_numpy(v).cuda() for k, v in ran.items()}
    ms = []
    for _ in range(max(1, args.fused_mocks // 4)):
        ng = int(min(gal["x"].size, g.uniform(5e5, 1.2e6)))
        ms.append((subsample(dg, ng), subsample(dr, min(ran["x"].size, 30 * ng))))
    del dg, dr
    out["boss_256"] = dict(workload=f"{len(ms)} BOSS-like mocks, 256^3 TSC, N_g in [5e5, 1.2e6] + 30x randoms",
                           **_fused_vs_single(fkp.Plan(svb.geometry(), BINS, want=want), ms, 3))
    return out


def _rel_diff(a, b, keys, den):
    """max |a - b| / max(|b|, den) over the entries where den is finite."""
    out = 0.0
    m = np.isfinite(den) & (den > 0)
    for k in keys:
        d = np.maximum(np.abs(b[k][m]), den[m])
        out = max(out, float(np.max(np.abs(a[k][m] - b[k][m]) / d)))
    return out


def run_batch(args):
    """The batched-mock workload: mocks drawn from a device-resident master
    catalog (1.2e6 galaxies and 30x randoms, the BOSS-like footprint with nbar
    scaled up): grid from {256, 384, 512}, N_g uniform in [5e5, 1.2e6] (a
    random subsample), randoms 30 N_g; each mock P_0,2,4 plus B_0 to k = 0.15
    (27 shells).  Batched: all mocks submitted to the request server at once
    (3 slots, plans pooled per grid, 3-way split tensor-core contraction).
    Plain: the per-mock path, one at a time on one stream, FP32 contraction.
    Reports mocks/s for both and, per mock, the largest difference between
    them (P_l graded by the raw monopole, B_0 by |T_0|/(N^3 N_T I_33) over
    triangles with N_T >= 100); the FP64 parity of each path is what
    tests/test_gpu_power.py and tests/test_gpu_bispectrum.py check."""
    import dataclasses

    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    base = mockgen.survey_boss(N=256)
    sv = dataclasses.replace(base, nbar_peak=base.nbar_peak * 1.2e6 / 7.0e5, random_ratio=30.0)
    gal, ran = mockgen.catalog(sv, args.seed + 500)
    dgal = {k: torch.from_numpy(v).cuda() for k, v in gal.items()}
    dran = {k: torch.from_numpy(v).cuda() for k, v in ran.items()}
    ngal, nran = gal["x"].size, ran["x"].size
    del gal, ran
    g = np.random.default_rng(args.seed + 300)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(args.seed + 301)
    want = fkp.FKP_P0 | fkp.FKP_P2 | fkp.FKP_P4 | fkp.FKP_B0
    bshells = (3, 3, 3, 27)
    mocks = []
    for _ in range(args.batch_mocks):
        N = int(g.choice([256, 384, 512]))
        ng = int(min(ngal, g.uniform(5e5, 1.2e6)))
        nr = min(nran, 30 * ng)
        gi = torch.sort(torch.randperm(ngal, device="cuda", generator=gen)[:ng]).values
        ri = torch.sort(torch.randperm(nran, device="cuda", generator=gen)[:nr]).values
        mocks.append(dict(geom=mockgen.survey_boss(N=N).geometry(),
                          gal={k: v[gi].contiguous() for k, v in dgal.items()},
                          ran={k: v[ri].contiguous() for k, v in dran.items()}, n_obj=ng + nr))
    del dgal, dran
    torch.cuda.synchronize()
    srv = fkp.Server(nslots=3)

    def submit_all():
        return [srv.submit(m["geom"], BINS, m["gal"], m["ran"], want=want, bshells=bshells,
                           contraction=fkp.FKP_CONTRACT_BF16X6) for m in mocks]

    for t in submit_all():  # plans and schedules for every grid
        srv.wait(t)
    t0 = time.perf_counter()
    served = [srv.wait(t) for t in submit_all()]
    wall_b = time.perf_counter() - t0
    srv.close()
    plans = {}
    for m in mocks:
        N = m["geom"]["N"]
        if N not in plans:
            plans[N] = fkp.Plan(m["geom"], BINS, bshells=bshells, want=want)
            plans[N].bispectrum(m["gal"], m["ran"], contraction=fkp.FKP_CONTRACT_FP32)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    plain = [plans[m["geom"]["N"]].bispectrum(m["gal"], m["ran"], contraction=fkp.FKP_CONTRACT_FP32) for m in mocks]
    wall_p = time.perf_counter() - t1
    for p in plans.values():
        p.close()
    dp, db = [], []
    for m, (ps, bs, _), (pp, bp) in zip(mocks, served, plain):
        dp.append(_rel_diff(ps, pp, ("P0", "P2", "P4"), np.abs(pp["mono_raw"])))
        N3 = float(m["geom"]["N"]) ** 3
        den = np.where(bp["NT"] >= 100, np.abs(bp["T0"]) / (N3 * np.maximum(bp["NT"], 1) * bp["I33"]), np.nan)
        db.append(_rel_diff(bs, bp, ("B0",), den))
    # each output against the FP64 oracle for a sample of the mocks (the
    # oracle takes tens of seconds per mock, so not all of them)
    vs_fp64 = []
    for j in range(min(args.batch_oracle_mocks, len(mocks))):
        m = mocks[j]
        hg = {k: v.cpu().numpy() for k, v in m["gal"].items()}
        hr = {k: v.cpu().numpy() for k, v in m["ran"].items()}
        vs_fp64.append(dict(mock=j, grid=m["geom"]["N"], **_vs_oracle(hg, hr, m["geom"], bshells, served[j][0],
                                                                      served[j][1], plain[j][1])))
    return {"workload": f"{len(mocks)} mocks: grids {{256,384,512}}, N_g in [5e5, 1.2e6] + 30x randoms (device "
                        "catalogs), P_0,2,4 + B_0 to k=0.15 (27 shells)",
            "unit": "mocks/s", "batched_mocks_per_s": len(mocks) / wall_b,
            "plain_mocks_per_s": len(mocks) / wall_p,
            "objects_per_mock_mean": float(np.mean([m["n_obj"] for m in mocks])),
            "batched_vs_plain_max_rel_diff": {"P": max(dp), "B0": max(db)},
            "per_mock_rel_diff_P": dp, "per_mock_rel_diff_B0": db, "per_mock_error_vs_fp64": vs_fp64}


def _vs_oracle(gal, ran, geom, bshells, p_served, b_served, b_plain):
    """Largest error of P_0,2,4 (graded by max(|P|, raw monopole)) and of B_0
    (graded by max(|B_0|, |T_0|/(N^3 N_T I_33)), N_T >= 100) of one mock's
    served and plain outputs against the FP64 oracle."""
    from oracle import bispectrum as ob
    from oracle import power as op
    N = int(geom["N"])
    Fl, Fwl, sc = op.survey_fields(gal, ran, geom, lmax=4, with_w2=True)
    ref = op.bin_power(Fl, geom, BINS, sc["I22"], sc["N0"])
    m = ref["nmodes"] > 0
    den = np.maximum(np.abs(ref["P0"][m]), np.abs(ref["mono_raw"][m]))
    eP = max(float(np.max(np.abs(p_served[k][m] - ref[k][m]) / np.maximum(np.abs(ref[k][m]), den)))
             for k in ("P0", "P2", "P4"))
    tri = [tuple(t) for t in b_served["tri"].astype(int)]
    g = np.random.default_rng(N)
    sample = sorted(tri[i] for i in g.permutation(len(tri))[:40])
    rb = ob.bispectrum_from_fields({0: Fl[0]}, {0: Fwl[0]}, sc, N, bshells, ells=(0,), tris=sample, cache_fields=8)
    idx = [tri.index(t) for t in sample]
    mm = rb["NT"] >= 100
    dB = np.maximum(np.abs(rb["B0"][mm]), np.abs(rb["T0"][mm]) / (float(N) ** 3 * rb["NT"][mm] * rb["I33"]))
    eB = {name: float(np.max(np.abs(b["B0"][idx][mm] - rb["B0"][mm]) / dB))
          for name, b in (("served_bf16x6", b_served), ("plain_fp32", b_plain))}
    return {"P_max_err": eP, "B0_max_err_40_triangles": eB}


def run_serve(args, gal, ran):
    """A stream of uneven requests shaped like the batched-mock workload:
    grid drawn from {256, 384, 512}, galaxies a random 50-100 % subsample of
    the 7e5-galaxy catalog, randoms 30x the galaxies, host (pinned) catalogs
    copied in by each request; half ask for P_0,2,4 + P_4b only, half also
    for B_0,2,4 to k = 0.2 (37 shells of 3 k_f) where the grid allows it
    (3 n_max < N), else to k = 0.15 (27 shells).  The served form runs the
    3-way split tensor-core contraction; the plain form is the sequential GPU
    path (one request at a time on one stream) with the FP32 CUDA-core
    contraction, both within the 1e-4 bar.  Reports p50/p99 latency
    (submission to result on the host) under Poisson arrivals and saturated
    mocks/s (all requests submitted at once) against the plain form."""
    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    g = np.random.default_rng(args.seed + 77)
    # the catalogs are in random order (galaxies shuffled, randoms drawn
    # independently), so a contiguous slice at a random offset is a random
    # subsample: every request is a view into one pinned copy of the catalogs
    pg = {k: torch.from_numpy(v).pin_memory() for k, v in gal.items()}
    pr = {k: torch.from_numpy(v).pin_memory() for k, v in ran.items()}
    reqs = []
    for i in range(args.serve_requests):
        N = int(g.choice([256, 384, 512]))
        ng = int(gal["x"].size * g.uniform(0.5, 1.0))
        nr = min(ran["x"].size, 30 * ng)
        og = int(g.integers(0, gal["x"].size - ng + 1))
        orr = int(g.integers(0, ran["x"].size - nr + 1))
        hg = {k: v[og:og + ng] for k, v in pg.items()}
        hr = {k: v[orr:orr + nr] for k, v in pr.items()}
        B = bool(i % 2)
        S = 37 if 3 * (3 * 37 + 1.5) < N else 27
        reqs.append(dict(geom=mockgen.survey_boss(N=N).geometry(), gal=hg, ran=hr, B=B, S=S, n_obj=ng + nr))
    pb = BINS

    def submit(srv, r):
        if r["B"]:
            return srv.submit(r["geom"], pb, r["gal"], r["ran"], want=BALL, bshells=(3, 3, 3, r["S"]),
                              contraction=fkp.FKP_CONTRACT_BF16X6)
        return srv.submit(r["geom"], pb, r["gal"], r["ran"])

    srv = fkp.Server(nslots=args.serve_slots)
    for t in [submit(srv, r) for r in reqs]:  # warm the plan pool and the kernels
        srv.wait(t)
    # Poisson arrivals
    arr = np.cumsum(g.exponential(1.0 / args.serve_rate, size=len(reqs)))
    t0 = time.perf_counter()
    tickets = []
    for a, r in zip(arr, reqs):
        dt = t0 + a - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(submit(srv, r))
    lat = [srv.wait(t)[2] for t in tickets]
    wall_poisson = time.perf_counter() - t0
    # saturated: everything at once
    t1 = time.perf_counter()
    ts = [submit(srv, r) for r in reqs]
    lat_sat = [srv.wait(t)[2] for t in ts]
    wall_sat = time.perf_counter() - t1
    st = srv.stats()
    srv.close()
    # plain sequential GPU path: one request at a time on one stream, plans
    # cached by geometry (made before the timed loop, as the server's pool is
    # warm before its timed stream)
    plans = {}

    def plan_for(r):
        key = (r["geom"]["N"], r["B"])
        if key not in plans:
            plans[key] = (fkp.Plan(r["geom"], pb, bshells=(3, 3, 3, r["S"]), want=BALL) if r["B"]
                          else fkp.Plan(r["geom"], pb))
        return plans[key]

    plain_reqs = reqs[:max(1, min(len(reqs), args.serve_plain_requests))]
    for r in plain_reqs:
        plan_for(r)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for r in plain_reqs:
        plan = plan_for(r)
        if r["B"]:
            plan.bispectrum(r["gal"], r["ran"], contraction=fkp.FKP_CONTRACT_FP32)
        else:
            plan.power(r["gal"], r["ran"])
    wall_seq = time.perf_counter() - t2
    for p in plans.values():
        p.close()
    n = len(reqs)
    return {"workload": f"{n} requests, grids {{256,384,512}}, 3.5e5-7e5 galaxies + 30x randoms (host catalogs), "
                        "half P_0,2,4+P_4b, half also B_0,2,4 (37 shells to k=0.2, 27 at 256^3); served: "
                        "3-way split bf16 tcgen05 contraction, plain: sequential FP32 contraction",
            "arrival_rate_per_s": args.serve_rate, "slots": args.serve_slots,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "poisson_wall_s": wall_poisson,
            "saturated_mocks_per_s": n / wall_sat, "saturated_p50_ms": float(np.percentile(lat_sat, 50)),
            "plain_sequential_mocks_per_s": len(plain_reqs) / wall_seq,
            "plain_sequential_requests": len(plain_reqs),
            "peak_running": st["peak_running"], "peak_bytes": int(st["peak_bytes"])}


# ---------------------------------------------------------------------------
# synthetic versions of the paper's experiments (--experiment; not part of the
# default run): many mocks that share one random catalog, the randoms
# gridded once onto the plan (fkp_plan_cache_randoms), galaxies generated on
# the host by a spawn pool while the GPU measures the previous mocks
# ---------------------------------------------------------------------------

def _gen_galaxies(task):
    import mockgen
    sv, seed = task
    return seed, mockgen.galaxies(sv, seed)


def _mock_stream(sv, seeds, workers):
    """Galaxy catalogs of the given seeds, generated in a spawn pool."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        for seed, gal in pool.imap(_gen_galaxies, [(sv, s) for s in seeds]):
            yield seed, gal


def experiment_p4b(args):
    """The two hexadecapole estimators over an ensemble of mocks (the analogue
    of Sec. III.A's comparison on the LasDamas and PTHalos mocks, Figs. 1-2):
    per k bin the bias ratio b_4 = <P_4b>/<P_4> and the cosmic-variance ratio
    sigma_4^2 = var(P_4b)/var(P_4), with the standard error of b_4.  BOSS-like
    mocks (512^3 TSC unless --grid), one random catalog (50x) for all."""
    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    sv = mockgen.survey_boss(N=args.grid, random_ratio=args.ran_ratio)
    ran = mockgen.randoms(sv, 0)
    plan = fkp.Plan(sv.geometry(), BINS)
    plan.cache_randoms({k: torch.from_numpy(v).cuda() for k, v in ran.items()})
    P4, P4b, k = [], [], None
    t0 = time.perf_counter()
    for seed, gal in _mock_stream(sv, range(1000, 1000 + args.experiment_mocks), args.experiment_workers):
        r = plan.power({kk: torch.from_numpy(v).cuda() for kk, v in gal.items()}, None)
        P4.append(r["P4"])
        P4b.append(r["P4b"])
        k = r["k_eff"]
    P4, P4b = np.array(P4), np.array(P4b)
    M = P4.shape[0]
    m4, m4b = P4.mean(0), P4b.mean(0)
    b4 = m4b / m4
    # standard error of the ratio of means (delta method with the covariance)
    cov = np.array([np.cov(P4[:, i], P4b[:, i]) for i in range(P4.shape[1])])
    se = np.abs(b4) * np.sqrt(np.maximum(cov[:, 0, 0] / m4 ** 2 + cov[:, 1, 1] / m4b ** 2
                                         - 2 * cov[:, 0, 1] / (m4 * m4b), 0.0) / M)
    return {"experiment": "P_4b vs P_4 over mocks (Sec. III.A, Figs. 1-2 analogue)",
            "workload": f"{M} BOSS-like mocks, {sv.N}^3 TSC, galaxies seeds 1000..{999 + M}, one random catalog "
                        f"({int(ran['x'].size)} randoms, cached on the plan)",
            "wall_s": time.perf_counter() - t0, "k": k.tolist(), "b4": b4.tolist(), "b4_se": se.tolist(),
            "sigma4_sq_ratio": (P4b.var(0, ddof=1) / P4.var(0, ddof=1)).tolist(),
            "mean_P4": m4.tolist(), "mean_P4b": m4b.tolist()}


def experiment_qell(args):
    """The reduced bispectrum multipoles Q^(l) = B_l/(P_0(k1) P_0(k2) +
    P_0(k2) P_0(k3) + P_0(k3) P_0(k1)) (eq. Qelldef) for k1 = 0.047 h/Mpc,
    k2 = 2 k1 as a function of the angle theta between k1 and k2 (the
    analogue of Sec. III.B's Fig. 3), averaged over mocks: 360^3 TSC, shells
    of 3 k_f, P_0 in bins that are the shells themselves; the l-th multipole
    is about the largest side (k1 >= k2 >= k3 order of the triangle)."""
    import torch

    import mockgen
    import paper_1506_02729_gb300 as fkp
    sv = mockgen.survey_boss(N=360, random_ratio=args.ran_ratio)
    kf = 2 * math.pi / sv.L
    bs = (3, 3, 3, 37)
    pb = (1.5 * kf, 3 * kf, 37)  # P bins = the bispectrum shells
    s1 = int(round(0.047 / (3 * kf))) - 1
    s2 = 2 * (s1 + 1) - 1        # centre exactly twice s1's
    ran = mockgen.randoms(sv, 0)
    plan = fkp.Plan(sv.geometry(), pb, bshells=bs, want=fkp.FKP_P0 | fkp.FKP_B0 | fkp.FKP_B2 | fkp.FKP_B4)
    plan.cache_randoms({k: torch.from_numpy(v).cuda() for k, v in ran.items()})
    rows, Q = None, []
    t0 = time.perf_counter()
    for seed, gal in _mock_stream(sv, range(2000, 2000 + args.experiment_mocks), args.experiment_workers):
        p, b = plan.bispectrum({kk: torch.from_numpy(v).cuda() for kk, v in gal.items()}, None,
                               contraction=fkp.FKP_CONTRACT_BF16X6)
        tri = b["tri"].astype(int)
        if rows is None:
            rows = [i for i, t in enumerate(tri) if s1 in t and s2 in t]
        P0 = p["P0"]
        q = []
        for i in rows:
            a, bb, c = tri[i]
            den = P0[a] * P0[bb] + P0[bb] * P0[c] + P0[c] * P0[a]
            q.append([b["B0"][i] / den, b["B2"][i] / den, b["B4"][i] / den])
        Q.append(q)
    Q = np.array(Q)
    cen = 3 * (np.arange(37) + 1) * kf
    out = []
    for j, i in enumerate(rows):
        sides = list(tri[i])
        rest = list(sides)
        rest.remove(s1)
        rest.remove(s2)
        s3 = rest[0]
        cth = (cen[s3] ** 2 - cen[s1] ** 2 - cen[s2] ** 2) / (2 * cen[s1] * cen[s2])
        out.append({"shells": [int(v) for v in sides], "theta_over_pi": float(np.arccos(np.clip(cth, -1, 1)) / np.pi),
                    "NT": int(b["NT"][i]), "Q0": float(Q[:, j, 0].mean()), "Q2": float(Q[:, j, 1].mean()),
                    "Q4": float(Q[:, j, 2].mean()), "Q0_se": float(Q[:, j, 0].std(ddof=1) / np.sqrt(len(Q))),
                    "Q2_se": float(Q[:, j, 1].std(ddof=1) / np.sqrt(len(Q))),
                    "Q4_se": float(Q[:, j, 2].std(ddof=1) / np.sqrt(len(Q)))})
    out.sort(key=lambda r: r["theta_over_pi"])
    return {"experiment": "Q^(l)(theta) for k1 = 0.047, k2 = 2 k1 (eq. Qelldef; Sec. III.B, Fig. 3 analogue)",
            "workload": f"{len(Q)} BOSS-like mocks, 360^3 TSC, 37 shells of 3 k_f, one cached random catalog",
            "k1": float(cen[s1]), "k2": float(cen[s2]), "wall_s": time.perf_counter() - t0, "triangles": out}


def main():
    args = parse()
    if args.experiment:
        out = {"p4b": experiment_p4b, "qell": experiment_qell}[args.experiment](args)
        print(json.dumps(out), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()

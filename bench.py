#!/usr/bin/env python
"""Throughput of the RKHS-BA hot path on GB300: pair-terms/s for
loss + gradient + Gauss-Newton blocks, measured on the global-mapping
workload (64 frames x 100k LiDAR points on a loop with loop closures, 516
frame pairs, 19-class labels stored as BF16, ell = 0.3 m, r_c = 0.9 m),
synthetic and seeded; the 8 x 20k multi-view registration and the 10 x 50k
sliding-window workloads are measured beside it.

One step = one pass of the whole hot path over the resident problem:
grid build of every frame, the evaluation at the initial poses (transform,
binning, pair kernel, FP64 assembly) and one Levenberg-Marquardt iteration
(Cholesky solve of the 6K x 6K system, SE(3) update, evaluation at the
candidate, accept/reject).  Pair-terms counted are those of the two
evaluations of the step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own replica (the path shards by problem;
there is no data-path collective), value = all pair-terms / max rank time.
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

METRIC = "pair-terms/s for RKHS-BA loss+grad+Hessian; served BA solves/s, p50/p99 latency"
UNIT = "pair-terms/s"
WORKLOAD = "mapping_64x100000"
SECONDARY = ("lidar_street_8x20000", "window_10x50000")
L2_FLUSH_BYTES = 256 << 20


PAIR_SOURCES = ("paper_2403_01254_gb300/csrc/pairs.cu", "paper_2403_01254_gb300/csrc/common.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_pairs_dram_traffic.json")


def pair_kernel_digest():
    """SHA-256 over the code of the pair kernel's sources (line comments and
    whitespace removed): a recorded DRAM traffic figure is reported only while
    the kernel is the one it was taken on."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in PAIR_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            code = re.sub(r"//[^\n]*", "", f.read())
        h.update(re.sub(r"\s+", "", code).encode())
    return h.hexdigest()


def recorded_traffic(workload_name):
    """dram__bytes_read.sum + dram__bytes_write.sum of one k_pairs launch from
    an ncu capture of this workload, or None when absent or stale."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(workload_name)
    if not ent or ent.get("source_sha256") != pair_kernel_digest():
        return None
    return ent.get("bytes_per_launch")


# Algorithmic FP32 work of one pair-term (what the method must do per pair
# inside r_c): d and |d|^2 (3 sub + 3 FMA), the exponent and one exp, the
# 19-term label dot (19 FMA) and the updates of the 28 edge moments: about 60
# FP32 instructions, 110 flops.  The roofline fraction is stated on this basis.
FLOPS_PER_PAIR = 110


def kernel_path(flat):
    """Which pair kernel serves the workload and where its arithmetic runs.
    Without colour the dense tile kernel evaluates every candidate x query
    element of a 32 x 32 batch: the cutoff test, the exponent and w = s k on
    the FP32 pipe (9 flops per element) and one ex2; the label products and
    the per-query moment sums on the tensor cores (mma.sync, BF16 or split
    FP16 operands, FP32 accumulation)."""
    if flat["color"]:
        return "bit-walk (colour): FP32 label dot and moment sums per pair on the FP32 pipe"
    return ("dense tile: test, exponent and weight on the FP32 pipe (9 flops per tested element), label "
            "products and moment sums on the tensor cores (mma.sync, %s operands)"
            % ("BF16 labels / split FP16 features" if flat["P"].get("sem_bf16", 0) else "split FP16"))


WORKLOADS = {
    # name: (generator, kwargs); the default is the headline workload
    "lidar_street_8x20000": ("lidar_street_problem", dict(seed=1434)),
    "plane_sphere_2x2000": ("plane_sphere_problem", dict(seed=1334)),
    "window_10x50000": ("window_problem", dict(seed=1534, window=10)),
    "mapping_64x100000": ("mapping_problem", dict(seed=1734)),
}


def workload(name=None):
    import scenes
    gen, kw = WORKLOADS[name or WORKLOAD]
    return getattr(scenes, gen)(**kw)


# ------------------------------------------------------------------ oracle --
def _oracle_edges(prob, name):
    """Frame pairs of the CPU samples: for the mapping workload the first
    odometry edge (0,1) and the first loop-closure edge (0,16); otherwise the
    first two edges (the only one of a single-edge problem)."""
    E = np.asarray(prob["edges"])
    if name.startswith("mapping"):
        return [0, int(np.nonzero(E[:, 1] - E[:, 0] > 7)[0][0])]
    return [0, 1] if len(E) > 1 else [0]


def _truncated(prob, e, n_b):
    """The problem with the second frame of edge e cut to its first n_b points."""
    b = int(np.asarray(prob["edges"])[e][1])
    sub = dict(prob, xyz=list(prob["xyz"]), sem=list(prob["sem"]) if prob.get("sem") is not None else None)
    sub["xyz"][b] = prob["xyz"][b][:n_b]
    if sub["sem"] is not None:
        sub["sem"][b] = prob["sem"][b][:n_b]
    return sub


def oracle_baseline(prob, name):
    """The FP64 oracle timed on the host cores on a bounded sample of the
    workload: every core (a spawned pool, each worker single-threaded, the
    edges' sums split over slices of frame b's points), and one core on a
    smaller sample.  Value = pair-terms / wall time."""
    from oracle.split_sum import evaluate_split, make_pool
    ids = _oracle_edges(prob, name)
    E = np.asarray(prob["edges"])
    T = prob["poses0"]
    cores = os.cpu_count() or 1
    with make_pool(cores) as pool:
        pool.submit(int, 0).result()                       # workers up before the clock starts
        r = evaluate_split(prob, T, ids, pool=pool)
    one_sub = _truncated(prob, ids[0], 8000)
    with make_pool(1) as pool:
        pool.submit(int, 0).result()
        r1 = evaluate_split(one_sub, T, [ids[0]], pool=pool)
    pairs = "+".join("(%d,%d)" % tuple(int(v) for v in E[e]) for e in ids)
    return dict(value=r["n_pairs"] / r["wall_s"], unit=UNIT, cores=r["workers"], kind="oracle",
                sample="edges %s of %s at the initial poses, full density (%d pair-terms, %.1f s wall on %d "
                       "processes)" % (pairs, name, r["n_pairs"], r["wall_s"], r["workers"]),
                single_core=dict(value=r1["n_pairs"] / r1["wall_s"], cores=1,
                                 sample="edge (%d,%d) of %s, first 8000 points of frame %d (%d pair-terms, %.1f s)"
                                        % (int(E[ids[0]][0]), int(E[ids[0]][1]), name, int(E[ids[0]][1]),
                                           r1["n_pairs"], r1["wall_s"])))


def reference_arm(args, rank):
    """The oracle as the reference arm: each step evaluates a bounded sample
    of the workload (edge (0,1), the first 16000 points of frame 1, at the
    initial poses) on every host core; warm-up steps first."""
    if rank != 0:
        return
    from oracle.split_sum import evaluate_split, make_pool
    prob = workload(args.workload)
    sub = _truncated(prob, 0, 16000)
    b = int(np.asarray(prob["edges"])[0][1])
    desc = ("edge (0,%d) of %s with the first 16000 points of frame %d, at the initial poses, "
            "on every host core" % (b, args.workload, b))
    cores = os.cpu_count() or 1
    tot_pairs, tot_s = 0, 0.0
    with make_pool(cores) as pool:
        pool.submit(int, 0).result()
        for _ in range(args.warmup):
            evaluate_split(sub, prob["poses0"], [0], slice_points=1000, pool=pool)
        for _ in range(args.steps):
            r = evaluate_split(sub, prob["poses0"], [0], slice_points=1000, pool=pool)
            tot_pairs += r["n_pairs"]
            tot_s += r["wall_s"]
    value = tot_pairs / tot_s
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * tot_s / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=args.workload, sample=desc),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores, kind="oracle", sample=desc),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        self.index = index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        self.t_start = self.t_end = None

    def mark(self, start):
        if start:
            self.t_start = time.time()
        else:
            self.t_end = time.time()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for ln in out.strip().splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append(dict(sm=float(parts[0]), smax=float(parts[1]), reasons=parts[3:]))
            except ValueError:
                continue
        if not rows:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=[], samples=0)
        # samples are ~100 ms apart; keep the ones that show the GPU under load
        loaded = [r for r in rows if r["sm"] > 0.5 * r["smax"]] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r["reasons"][1:5])
                          if v.strip().lower() == "active"})
        return dict(sm_mhz=statistics.median(r["sm"] for r in loaded),
                    sm_max_mhz=max(r["smax"] for r in rows), reasons=reasons,
                    samples=len(loaded))


# -------------------------------------------------------------------- ours --
def replica_throughput(ms_local, pairs_per_step, steps, world, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    pairs_per_step x steps pair-terms; the job time is the slowest rank's
    (all_reduce MAX over the process group when world > 1)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return pairs_per_step * steps * world / (ms_max / 1e3), ms_max


def _flat_inputs(prob):
    K = len(prob["xyz"])
    sem_dim = prob["sem"][0].shape[1]
    P = prob["params"]
    color = prob.get("rgb") is not None and P.get("ell_color", 0.0) > 0
    return dict(
        K=K, sem_dim=sem_dim, P=P, color=color,
        n_points=np.array([len(x) for x in prob["xyz"]], np.int64),
        xyz=np.ascontiguousarray(np.concatenate(prob["xyz"])),
        sem=np.ascontiguousarray(np.concatenate(prob["sem"]).astype(np.float32)),
        rgb=np.ascontiguousarray(np.concatenate(prob["rgb"]).astype(np.float32)) if color else None,
        poses0=np.ascontiguousarray(prob["poses0"].reshape(K * 16)),
        edges=np.asarray(prob["edges"], np.int32))


def measure_device(pk, rb, prob, steps, warmup, dev, stream, flush, world=1, clocks_index=None, autotune=False,
                   unit_queries=None):
    """Time `steps` bench steps of the resident problem with CUDA events on
    the library's stream (L2 flushed between steps, outside the events);
    phase times from the library's own events.  With autotune the library's
    autotuner first times every pair-stage setting on this problem and the
    fastest is used.  Returns pair-terms per step, summed step time, phase
    times, launch count, clock samples and the tuning."""
    import torch
    f = _flat_inputs(prob)
    P = f["P"]
    params = pk.make_params(P["ell"], P["cutoff_mult"], P["sigma"], P.get("ell_color", 0.0), f["sem_dim"],
                            P.get("sem_bf16", 0), max_iters=1000)
    xyz_d = torch.from_numpy(f["xyz"]).to(dev)
    sem_d = torch.from_numpy(f["sem"]).to(dev)
    rgb_d = torch.from_numpy(f["rgb"]).to(dev) if f["color"] else None
    poses_d = torch.from_numpy(f["poses0"]).to(dev)
    torch.cuda.synchronize()
    tuning = None
    if autotune:
        best, table = rb.rkhsba_autotune(f["n_points"], xyz_d.data_ptr(), sem_d.data_ptr(),
                                         rgb_d.data_ptr() if f["color"] else None, f["edges"], params,
                                         f["poses0"], stream.cuda_stream, reps=2, on_device=True)
        params.cell_scale = best["cell_scale"]
        tuning = dict(chosen=best, table=table, timed="one evaluation (binning + pair stage + assembly), "
                                                      "mean of 2 after 1 untimed, CUDA events")
    ctx = pk.rkhsba_create_device(f["n_points"], xyz_d.data_ptr(), sem_d.data_ptr(),
                                  rgb_d.data_ptr() if f["color"] else None, f["edges"], params, stream.cuda_stream)
    if tuning:
        rb.rkhsba_set_tuning(ctx, tuning["chosen"]["unit_queries"], tuning["chosen"]["ctas_per_sm"])
    elif unit_queries:
        # a fixed setting (e.g. the one the autotuner picks, for a profiler run)
        rb.rkhsba_set_tuning(ctx, unit_queries, 0)
        tuning = dict(chosen=dict(cell_scale=1.0, unit_queries=unit_queries, ctas_per_sm=0, ms=None), table=None,
                      timed="set with --unit-queries, not autotuned")

    def step():
        rb.rkhsba_rebuild(ctx)
        rb.rkhsba_set_poses_device(ctx, poses_d.data_ptr())
        rb.rkhsba_iterate(ctx, 1)

    try:
        with torch.cuda.stream(stream):
            for _ in range(max(warmup, 1)):
                flush.zero_()
                step()
        stream.synchronize()
        _, st = rb.rkhsba_get_state(ctx, f["K"])
        pairs_per_step = st["pair_terms"]
        clocks = ClockSampler(clocks_index) if clocks_index is not None else None
        if clocks:
            time.sleep(0.3)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        rb.rkhsba_profile(ctx, 1)
        n_launch0 = pk.rkhsba_launch_count()
        if clocks:
            clocks.mark(True)
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.zero_()                      # L2 flush between steps, outside the events
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        if clocks:
            clocks.mark(False)
        if world > 1:
            torch.distributed.barrier()
        n_launch = pk.rkhsba_launch_count() - n_launch0
        prof = rb.rkhsba_profile(ctx, 0, read=True)
        clk = clocks.stop() if clocks else None
    finally:
        rb.rkhsba_destroy(ctx)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    return dict(pairs_per_step=int(pairs_per_step), ms=ms, prof=prof, launches=int(n_launch), clocks=clk,
                flat=f, tuning=tuning, params=params)


def measured_hbm_gbs():
    """The measured copy bandwidth of the GB300 (MEASURED_PEAKS.json, a
    STREAM-style copy), else 6.8 TB/s from an earlier copy measurement on a
    GB300, and which of the two it is."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError, TypeError):
        return 6800.0, "fallback"


def label_row_bytes(sem_dim, bf16):
    """Bytes of one stored label row (FP32 rows padded to 4..32 floats, BF16
    rows to 8..32 values)."""
    if sem_dim <= 0:
        return 0
    pads = (8, 16, 24, 32) if bf16 else (4, 8, 12, 16, 20, 24, 32)
    pad = next((p for p in pads if sem_dim <= p), pads[-1])
    return pad * (2 if bf16 else 4)


def pair_bounds(flat, pair_terms_per_launch, peak_tflops):
    """Both roofline bounds of the pair kernel in pair-terms/s: FP32 issue
    (peak / 110 flops per pair-term) and HBM (every point of both frames of
    every edge read once per launch: 16 B of position + its label row, at the
    measured copy bandwidth).  The lower one bounds the kernel."""
    n = flat["n_points"]
    E = np.asarray(flat["edges"])
    row = 16 + label_row_bytes(flat["sem_dim"], flat["P"].get("sem_bf16", 0)) + (16 if flat["color"] else 0)
    alg_bytes = float(sum(int(n[a]) + int(n[b]) for a, b in E)) * row
    gbs, src = measured_hbm_gbs()
    hbm = pair_terms_per_launch / (alg_bytes / (gbs * 1e9)) if alg_bytes > 0 else None
    fp32 = peak_tflops * 1e12 / FLOPS_PER_PAIR
    return dict(fp32_pair_terms_per_s=fp32, hbm_pair_terms_per_s=hbm, hbm_gbs=gbs, hbm_source=src,
                algorithmic_bytes_per_launch=alg_bytes, lower="fp32" if hbm is None or fp32 <= hbm else "hbm")


def roofline_of(name, m, steps, dev, sm_max):
    """Roofline of the dominant kernel (the pair kernel, bound by instruction
    issue): achieved = algorithmic flops (110 per pair-term) of the
    pair-terms one launch processes / that launch's CUDA-event time; peak =
    SMs x 128 FP32 lanes x 2 flop x clock."""
    import torch
    pair_ms, pair_n = m["prof"]["pairs"]
    props = torch.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    terms = m["pairs_per_step"] * steps
    achieved = terms * FLOPS_PER_PAIR / (pair_ms / 1e3) / 1e12 if pair_ms > 0 else None
    return dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                frac=(achieved / peak) if achieved else None, traffic=recorded_traffic(name),
                kernel="k_pairs", flops_per_pair_term=FLOPS_PER_PAIR,
                peak_basis="%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (nominal unit counts; no measured FP32 peak)"
                           % (props.multi_processor_count, sm_max),
                kernel_path=kernel_path(m["flat"]),
                pair_terms_per_launch=m["pairs_per_step"] / 2,
                pair_kernel_ms_per_launch=pair_ms / max(pair_n, 1),
                pair_terms_per_s_in_kernel=terms / (pair_ms / 1e3) if pair_ms > 0 else None,
                bounds=pair_bounds(m["flat"], m["pairs_per_step"] / 2, peak),
                phases_ms_per_step={k: v[0] / steps for k, v in m["prof"].items()})


def measure_e2e(pk, rb, f, stream, n_steps, tuning=None):
    """Same metric through the public C ABI from pinned HOST buffers: each
    step is rkhsba_create (H2D of points and labels, grid build) +
    rkhsba_solve with max_iters 1 (two evaluations, D2H of the poses) +
    rkhsba_destroy, timed on the host around synchronous calls."""
    import torch
    P = f["P"]

    def pinned(a, dt):
        if a is None:
            return None
        out = torch.empty(a.shape, dtype=dt, pin_memory=True).numpy()
        out[:] = a
        return out
    xyz_p = pinned(f["xyz"], torch.float64)
    sem_p = pinned(f["sem"], torch.float32)
    rgb_p = pinned(f["rgb"], torch.float32)
    pos_p = pinned(f["poses0"], torch.float64)
    params1 = pk.make_params(P["ell"], P["cutoff_mult"], P["sigma"], P.get("ell_color", 0.0), f["sem_dim"],
                             P.get("sem_bf16", 0), max_iters=1,
                             cell_scale=tuning["cell_scale"] if tuning else 1.0)
    pairs, secs = 0, 0.0
    for k in range(n_steps + 2):
        pos_p[:] = f["poses0"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = rb.rkhsba_create_flat(f["n_points"], xyz_p, sem_p, rgb_p, f["edges"], params1, stream.cuda_stream)
        if tuning:
            rb.rkhsba_set_tuning(c2, tuning["unit_queries"], tuning["ctas_per_sm"])
        T, info = rb.rkhsba_solve(c2, pos_p, f["K"])
        rb.rkhsba_destroy(c2)
        dt = time.perf_counter() - t0
        if k >= 2:
            pairs += info["pair_terms"]
            secs += dt
    h2d = (f["xyz"].nbytes + f["sem"].nbytes + (f["rgb"].nbytes if f["color"] else 0) + f["poses0"].nbytes +
           f["edges"].nbytes + f["n_points"].nbytes)
    return dict(value=pairs / secs, unit=UNIT, h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(f["poses0"].nbytes + 64), steps=n_steps,
                step="create (H2D + grids) + solve with max_iters 1 + destroy" +
                     (", with the autotuned setting" if tuning else ""))


def ours(args, rank, world, local_rank):
    import torch

    import paper_2403_01254_gb300 as pk
    from paper_2403_01254_gb300 import rkhsba as rb

    prob = workload(args.workload)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before the first CUDA call; the oracle runs in spawned processes
        cpu_base = oracle_baseline(prob, args.workload)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pk.load()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    m = measure_device(pk, rb, prob, args.steps, args.warmup, dev, stream, flush, world, clocks_index=local_rank,
                       autotune=not args.no_autotune and not args.unit_queries, unit_queries=args.unit_queries)
    value, ms_max = replica_throughput(m["ms"], m["pairs_per_step"], args.steps, world, dev)
    clk = m["clocks"]
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    roofline = roofline_of(args.workload, m, args.steps, dev, sm_max)
    f = m["flat"]

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(pk, rb, f, stream, max(3, min(args.steps, 20)),
                          m["tuning"]["chosen"] if m["tuning"] else None)

    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary and args.workload == WORKLOAD:
        secondary = {}
        for name in SECONDARY:
            p2 = workload(name)
            steps2 = 50
            m2 = measure_device(pk, rb, p2, steps2, 5, dev, stream, flush, autotune=not args.no_autotune)
            secondary[name] = dict(
                value=m2["pairs_per_step"] * steps2 / (m2["ms"] / 1e3), unit=UNIT, steps=steps2,
                ms_per_step=m2["ms"] / steps2, pair_terms_per_step=m2["pairs_per_step"],
                roofline=roofline_of(name, m2, steps2, dev, sm_max),
                tuning=m2["tuning"]["chosen"] if m2["tuning"] else None)
    serve = None
    if rank == 0 and world == 1 and not args.no_serving and args.workload == WORKLOAD:
        serve = serving(pk)
    funcs = None
    if rank == 0 and world == 1 and not args.no_functions and args.workload == WORKLOAD:
        funcs = function_space(pk, workload(SECONDARY[0]))

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_max / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload=args.workload, frames=f["K"], points=int(f["n_points"].sum()),
                                edges=len(f["edges"]), sem_dim=f["sem_dim"],
                                labels="bf16" if f["P"].get("sem_bf16", 0) else "f32", ell=f["P"]["ell"],
                                pair_terms_per_step=int(m["pairs_per_step"]),
                                l2="256 MiB buffer written between steps, outside the timed events",
                                step="grid build + evaluation + one LM iteration (2 evaluations)",
                                parallelism="replicas" if world > 1 else "single GPU",
                                tuning=m["tuning"]["chosen"] if m["tuning"] else "default (untuned)"),
                    autotune=m["tuning"],
                    roofline=roofline, cpu_baseline=cpu_base, e2e=e2e, gpu_launches=m["launches"],
                    clocks=clk, secondary=secondary, serving=serve, functions=funcs)
        print(json.dumps(line), flush=True)


def function_space(pk, prob):
    """Latency of the function-space calls (host wall time around the
    synchronous C-ABI calls, median of repeats):
      - two-view global registration of Sec. VI-A on the object-pair scene
        (90 deg about a random axis, 0.5 m, 12.5% outliers and cropping, part
        labels) at 1000-8000 points per scan: the 60-rotation search, and the
        search followed by the LM solve at ell = 0.1, 0.05, 0.03;
      - inner products, distances and cosines of every edge of the bench
        workload (the self terms cached after the first call);
      - one evaluation of the bench workload with the top-8 neighbour limit
        and with semantic pruning at 0.1;
      - the lengthscale-decay loop on a 4-frame x 5000-point LiDAR problem."""
    import scenes

    def med(f, reps):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            out = f()
            ts.append(time.perf_counter() - t0)
        return 1e3 * float(np.median(ts)), out

    reg = []
    for n in (1000, 2000, 4000, 8000):
        p = scenes.object_pair_problem(seed=300 + n, angle_deg=90.0, n=n, outlier_ratio=0.125, crop_ratio=0.125,
                                       ell=0.1, labels=True)
        g = pk.Problem.from_scene(p)
        try:
            g.rotation_search(0, 1, p["poses0"])
            ms_search, out = med(lambda: g.rotation_search(0, 1, p["poses0"]), 5)
        finally:
            g.close()

        def full():
            T = np.stack([np.eye(4), out["best_pose"]])
            for ell in (0.1, 0.05, 0.03):
                h = pk.Problem.from_scene(p, ell=ell, max_iters=40)
                try:
                    T, _ = h.solve(T)
                finally:
                    h.close()
            return T
        ms_full, T = med(full, 3)
        E = np.linalg.inv(p["poses_gt"][1]) @ T[1]
        rot_err = float(np.arccos(np.clip((np.trace(E[:3, :3]) - 1) / 2, -1, 1)))
        reg.append(dict(points=n, search_ms=ms_search, search_plus_lm_ms=ms_full, rot_err_rad=rot_err))

    g = pk.Problem.from_scene(prob)
    try:
        g.inner_products(prob["poses0"])
        ms_ip, _ = med(lambda: g.inner_products(prob["poses0"]), 10)
    finally:
        g.close()
    variants = {}
    for name, over in (("top_8", dict(top_k=8)), ("sem_min_0.1", dict(sem_min=0.1))):
        g = pk.Problem.from_scene(prob, **over)
        try:
            g.eval(prob["poses0"], want_H=False)
            ms_v, out_v = med(lambda: g.eval(prob["poses0"], want_H=False), 5)
        finally:
            g.close()
        variants[name] = dict(eval_ms=ms_v, pair_terms=int(out_v["n_pairs"]))
    small = scenes.lidar_street_problem(seed=1435, n_frames=4, n_points=5000)
    g = pk.Problem.from_scene(small, max_iters=30)
    try:
        ms_decay, (T, info) = med(lambda: g.solve_ell_decay(small["poses0"], decay=0.2, ell_min=0.1,
                                                              max_outer=5), 3)
    finally:
        g.close()
    return dict(two_view_registration=reg, inner_products_ms=ms_ip, sparse_sum_variants=variants,
                ell_decay=dict(problem="lidar 4x5000", ms=ms_decay, levels=info["levels"],
                               ell=[float(x) for x in info["ell"]]),
                timing="host wall time around synchronous calls, median")


def _pose_diff(Ta, Tb):
    """Largest rotation angle (rad) and translation (m) between two pose sets."""
    dr = dt = 0.0
    for A, B in zip(Ta, Tb):
        E = np.linalg.inv(B) @ A
        c = np.clip((np.trace(E[:3, :3]) - 1.0) / 2.0, -1.0, 1.0)
        dr = max(dr, float(np.arccos(c)))
        dt = max(dt, float(np.linalg.norm(E[:3, 3])))
    return dr, dt


def serving(pk, seed=1634, n_requests=200, pool_size=50, max_iters=30, loads=(0.5, 1.0, 1.5)):
    """Served BA solves: a Poisson stream of n_requests requests (2-10 frames x
    5k-100k LiDAR points, log-uniform, 19-class labels) drawn in turn from
    pool_size generated problems, at several loads (x the measured plain
    single-stream capacity).  Served form: the request server in batched
    mode (continuous batching, one pair launch per round over every in-flight
    request that is ready, BF16 labels on the device, up to 8 in flight); at
    load 1 and at capacity also the server with per-request streams, and at
    capacity the batched server with autotuning (tuned beforehand on one pool
    request of each workload class).  Plain form: one request at a time through rkhsba_create +
    rkhsba_solve with FP32 labels.  Accuracy: the served (batched) poses of
    every pool problem against the plain FP32 poses of the same problem (both
    run max_iters LM iterations at most)."""
    import threading

    import scenes
    specs = scenes.request_stream(seed=seed, n_requests=n_requests)
    pool = []
    for sp in specs[:pool_size]:
        p = scenes.lidar_street_problem(seed=sp["seed"], n_frames=sp["n_frames"],
                                        n_points=sp["n_points"], sem_bf16=1)
        p["params"] = dict(p["params"], max_iters=max_iters)
        pool.append(p)
    order = [i % pool_size for i in range(n_requests)]
    plain_res, served_res = {}, {}

    def plain_solve(i):
        g = pk.Problem.from_scene(pool[i], sem_bf16=0)
        try:
            T, info = g.solve(pool[i]["poses0"])
        finally:
            g.close()
        plain_res.setdefault(i, T)
        return T, info

    def pct(x, q):
        return float(np.percentile(np.asarray(x), q))

    # plain single-stream service times (capacity) over the pool
    plain_solve(0)
    svc = []
    for i in range(pool_size):
        t0 = time.perf_counter()
        plain_solve(i)
        svc.append(time.perf_counter() - t0)
    mean_svc = sum(svc[order[i]] for i in range(n_requests)) / n_requests

    def run_served(arrivals, server=None, **kw):
        srv = server or pk.Server(max_inflight=8, **kw)
        lat, done_t = [None] * n_requests, [None] * n_requests
        tickets = [None] * n_requests
        fail = []

        def poller():
            for i in range(n_requests):
                while tickets[i] is None:
                    time.sleep(0.0002)
                r = srv.poll(tickets[i], timeout_ms=-1)
                done_t[i] = time.perf_counter()
                lat[i] = r[1]["latency_ms"]
                if r[1]["state"] != "finished":
                    fail.append(r[1])
                elif server is not None:
                    served_res.setdefault(order[i], r[0])

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        for i in range(n_requests):
            if arrivals is not None:
                dt = t0 + arrivals[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            tickets[i] = srv.submit(pool[order[i]])
        th.join()
        if server is None:
            srv.close()
        wall = max(done_t) - t0
        return dict(solves_per_s=n_requests / wall, p50_ms=pct(lat, 50), p99_ms=pct(lat, 99), failed=len(fail))

    def run_plain(arrivals):
        lat = []
        t0 = time.perf_counter()
        fin = t0
        for i in range(n_requests):
            arr = t0 + (arrivals[i] if arrivals is not None else 0.0)
            now = time.perf_counter()
            if now < arr:
                time.sleep(arr - now)
            plain_solve(order[i])
            fin = time.perf_counter()
            lat.append(1e3 * (fin - arr))
        return dict(solves_per_s=n_requests / (fin - t0), p50_ms=pct(lat, 50), p99_ms=pct(lat, 99))

    rng = np.random.default_rng(seed)
    sweep = []
    # one batched server for every run, warmed by one request; an autotuned
    # one, warmed by one request of every workload class it will meet
    srv_b = pk.Server(max_inflight=8, mode="batched")
    srv_b.poll(srv_b.submit(pool[0]), timeout_ms=-1)
    srv_t = pk.Server(max_inflight=8, mode="batched", autotune=True)
    seen = set()
    for p in pool:
        per_frame = sum(len(x) for x in p["xyz"]) / len(p["xyz"])
        cls = 0 if per_frame < 16384 else (1 if per_frame < 65536 else 2)
        if cls not in seen:
            seen.add(cls)
            srv_t.poll(srv_t.submit(p), timeout_ms=-1)
    try:
        for load in loads:
            rate = load / mean_svc
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
            ent = dict(load_factor=load, arrival_rate_per_s=rate, served=run_served(arrivals, server=srv_b),
                       plain_fp32_single=run_plain(arrivals))
            if load == 1.0:
                ent["served_per_request_streams"] = run_served(arrivals, mode="per_request")
            sweep.append(ent)
        capacity = dict(served=run_served(None, server=srv_b)["solves_per_s"],
                        served_per_request_streams=run_served(None, mode="per_request")["solves_per_s"],
                        served_autotuned=run_served(None, server=srv_t)["solves_per_s"],
                        plain_fp32_single=run_plain(None)["solves_per_s"])
    finally:
        srv_b.close()
        srv_t.close()
    diffs = [_pose_diff(served_res[i], plain_res[i]) for i in sorted(served_res) if i in plain_res]
    accuracy = dict(compared=len(diffs), max_rot_rad=max(d[0] for d in diffs) if diffs else None,
                    max_trans_m=max(d[1] for d in diffs) if diffs else None, tolerance=1e-4,
                    against="plain FP32-label GPU solve of the same problem (same LM, max_iters each)")
    return dict(metric="served BA solves/s, p50/p99 latency", requests=n_requests, pool=pool_size,
                max_iters=max_iters, mean_single_stream_service_ms=1e3 * mean_svc,
                pool_frames_points=[[len(p["xyz"]), int(sum(len(x) for x in p["xyz"]))] for p in pool],
                loads=sweep, capacity_solves_per_s=capacity, accuracy=accuracy,
                note="solves/s and latencies (submit to result) under Poisson arrivals at load_factor x the plain "
                     "single-stream capacity; capacity with every request queued at once")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-functions", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="measure the default pair-stage setting")
    ap.add_argument("--unit-queries", type=int, default=0,
                    help="measure this unit size (queries per warp unit) instead of autotuning")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="other workloads of the paper's shapes (the default is the headline workload)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

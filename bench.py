#!/usr/bin/env python
"""Throughput of the RKHS-BA hot path on GB300: pair-terms/s for
loss + gradient + Gauss-Newton blocks, measured on the 8-frame x 20k-point
LiDAR multi-view registration workload (28 frame pairs, 19-class FP32 label
distributions, ell = 0.3 m, r_c = 0.9 m), synthetic and seeded.

One step = one pass of the whole hot path over the resident problem:
grid build of every frame, the evaluation at the initial poses (transform,
binning, pair kernel, FP64 assembly) and one Levenberg-Marquardt iteration
(Cholesky solve, SE(3) update, evaluation at the candidate, accept/reject).
Pair-terms counted are those of the two evaluations of the step.

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
WORKLOAD = "lidar_street_8x20000"
L2_FLUSH_BYTES = 256 << 20


PAIR_SOURCES = ("paper_2403_01254_gb300/csrc/pairs.cu", "paper_2403_01254_gb300/csrc/common.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_pairs_dram_traffic.json")


def pair_kernel_digest():
    """SHA-256 over the sources of the pair kernel: a recorded DRAM traffic
    figure is reported only while the kernel is the one it was taken on."""
    import hashlib
    h = hashlib.sha256()
    for rel in PAIR_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
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


def flops_per_pair(sem_dim, color):
    """Algorithmic FP32 flops of one pair-term (FMA = 2): d (3), |d|^2 (5),
    exponent (1), label dot (2 D), w = s k (1), sums W, D, Q (1 + 3 + 3 + 12);
    colour factor adds 9."""
    return 29 + 2 * sem_dim + (9 if color else 0)


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
def oracle_sample(kind):
    """Run the FP64 oracle on a bounded sample of the workload (CPU only)."""
    import oracle
    prob = workload()
    if kind == "baseline":
        # two full frame pairs (0,1) and (0,2) at the initial poses
        sub = dict(prob, edges=np.asarray(prob["edges"])[[0, 1]])
        desc = "edges (0,1),(0,2) of the 8x20k workload at the initial poses"
    else:
        # frame pair (0,1), every 4th point of frame 1
        sub = dict(prob, edges=np.asarray(prob["edges"])[[0]])
        sub["xyz"] = list(prob["xyz"])
        sub["sem"] = list(prob["sem"])
        sub["xyz"][1] = prob["xyz"][1][::4]
        sub["sem"][1] = prob["sem"][1][::4]
        desc = "edge (0,1) of the 8x20k workload with every 4th point of frame 1"
    t0 = time.perf_counter()
    r = oracle.evaluate(sub, prob["poses0"])
    dt = time.perf_counter() - t0
    return dict(pairs=int(r["n_pairs"]), seconds=dt, sample=desc)


def run_oracle_subprocess(kind):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", kind],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def reference_arm(args, rank):
    if rank != 0:
        return
    env_cores = 1
    # warm-up steps, then K timed steps, each a bounded sample on 1 host core
    for _ in range(args.warmup):
        run_oracle_subprocess("step")
    tot_pairs, tot_s = 0, 0.0
    desc = ""
    for _ in range(args.steps):
        r = run_oracle_subprocess("step")
        tot_pairs += r["pairs"]
        tot_s += r["seconds"]
        desc = r["sample"]
    value = tot_pairs / tot_s
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * tot_s / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(workload=WORKLOAD, sample=desc),
                cpu_baseline=dict(value=value, unit=UNIT, cores=env_cores, kind="oracle",
                                  sample=desc),
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


def ours(args, rank, world, local_rank):
    import torch

    import paper_2403_01254_gb300 as pk
    from paper_2403_01254_gb300 import rkhsba as rb

    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before the first CUDA call: the oracle runs in a fresh process
        cb = run_oracle_subprocess("baseline")
        cpu_base = dict(value=cb["pairs"] / cb["seconds"], unit=UNIT, cores=1, kind="oracle",
                        sample=cb["sample"] + " (%d pair-terms, %.1f s)" % (cb["pairs"], cb["seconds"]))

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pk.load()
    prob = workload(args.workload)
    K = len(prob["xyz"])
    sem_dim = prob["sem"][0].shape[1]
    n_points = np.array([len(x) for x in prob["xyz"]], np.int64)
    xyz_h = np.ascontiguousarray(np.concatenate(prob["xyz"]))
    sem_h = np.ascontiguousarray(np.concatenate(prob["sem"]).astype(np.float32))
    poses0 = np.ascontiguousarray(prob["poses0"].reshape(K * 16))
    edges = np.asarray(prob["edges"], np.int32)
    P = prob["params"]
    color = prob.get("rgb") is not None and P.get("ell_color", 0.0) > 0
    rgb_h = np.ascontiguousarray(np.concatenate(prob["rgb"]).astype(np.float32)) if color else None
    params = pk.make_params(P["ell"], P["cutoff_mult"], P["sigma"], P.get("ell_color", 0.0), sem_dim,
                            P.get("sem_bf16", 0), max_iters=1000)
    stream = torch.cuda.Stream(device=dev)
    xyz_d = torch.from_numpy(xyz_h).to(dev)
    sem_d = torch.from_numpy(sem_h).to(dev)
    rgb_d = torch.from_numpy(rgb_h).to(dev) if color else None
    poses_d = torch.from_numpy(poses0).to(dev)
    torch.cuda.synchronize()
    ctx = pk.rkhsba_create_device(n_points, xyz_d.data_ptr(), sem_d.data_ptr(),
                                  rgb_d.data_ptr() if color else None, edges, params, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        rb.rkhsba_rebuild(ctx)
        rb.rkhsba_set_poses_device(ctx, poses_d.data_ptr())
        rb.rkhsba_iterate(ctx, 1)

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            flush.zero_()
            step()
    stream.synchronize()
    _, st = rb.rkhsba_get_state(ctx, K)
    pairs_per_step = st["pair_terms"]

    clocks = ClockSampler(local_rank)
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    rb.rkhsba_profile(ctx, 1)
    n_launch0 = pk.rkhsba_launch_count()
    clocks.mark(True)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()                      # L2 flush between steps, outside the events
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark(False)
    if world > 1:
        torch.distributed.barrier()
    n_launch = pk.rkhsba_launch_count() - n_launch0
    prof = rb.rkhsba_profile(ctx, 0, read=True)
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    value, ms_max = replica_throughput(ms, pairs_per_step, args.steps, world, dev)

    # roofline of the dominant kernel (the pair kernel): FP32 arithmetic
    pair_ms, pair_n = prof["pairs"]
    fl = flops_per_pair(sem_dim, color)
    achieved = pairs_per_step * args.steps * fl / (pair_ms / 1e3) / 1e12 if pair_ms > 0 else None
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    roofline = dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                    frac=(achieved / peak) if achieved else None, traffic=recorded_traffic(args.workload),
                    kernel="k_pairs", flops_per_pair_term=fl,
                    peak_basis="%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz" %
                               (props.multi_processor_count, sm_max),
                    pair_kernel_ms_per_launch=pair_ms / max(pair_n, 1),
                    phases_ms_per_step={k: v[0] / args.steps for k, v in prof.items()})
    rb.rkhsba_destroy(ctx)

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        xyz_p = torch.empty(xyz_h.shape, dtype=torch.float64, pin_memory=True).numpy()
        sem_p = torch.empty(sem_h.shape, dtype=torch.float32, pin_memory=True).numpy()
        pos_p = torch.empty(poses0.shape, dtype=torch.float64, pin_memory=True).numpy()
        xyz_p[:] = xyz_h
        sem_p[:] = sem_h
        params1 = pk.make_params(P["ell"], P["cutoff_mult"], P["sigma"], P.get("ell_color", 0.0),
                                 sem_dim, P.get("sem_bf16", 0), max_iters=1)
        rgb_p = None
        if color:
            rgb_p = torch.empty(rgb_h.shape, dtype=torch.float32, pin_memory=True).numpy()
            rgb_p[:] = rgb_h
        n_e2e = max(3, min(args.steps, 20))
        e2e_pairs, e2e_s = 0, 0.0
        for k in range(n_e2e + 2):
            pos_p[:] = poses0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = rb.rkhsba_create_flat(n_points, xyz_p, sem_p, rgb_p, edges, params1,
                                       stream.cuda_stream)
            T, info = rb.rkhsba_solve(c2, pos_p, K)
            rb.rkhsba_destroy(c2)
            dt = time.perf_counter() - t0
            if k >= 2:
                e2e_pairs += info["pair_terms"]
                e2e_s += dt
        h2d = (xyz_h.nbytes + sem_h.nbytes + (rgb_h.nbytes if color else 0) + poses0.nbytes +
               edges.nbytes + n_points.nbytes)
        e2e = dict(value=e2e_pairs / e2e_s, unit=UNIT, h2d_bytes_per_step=int(h2d),
                   d2h_bytes_per_step=int(poses0.nbytes + 64), steps=n_e2e,
                   step="create (H2D + grids) + solve with max_iters 1 + destroy")

    serve = None
    if rank == 0 and world == 1 and not args.no_serving and args.workload == WORKLOAD:
        serve = serving(pk)
    funcs = None
    if rank == 0 and world == 1 and not args.no_functions and args.workload == WORKLOAD:
        funcs = function_space(pk, prob)

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=ms_max / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload=args.workload, frames=K, points=int(n_points.sum()),
                                edges=len(edges), sem_dim=sem_dim, ell=P["ell"],
                                pair_terms_per_step=int(pairs_per_step),
                                l2="256 MiB buffer written between steps, outside the timed events",
                                step="grid build + evaluation + one LM iteration (2 evaluations)",
                                parallelism="replicas" if world > 1 else "single GPU"),
                    roofline=roofline, cpu_baseline=cpu_base, e2e=e2e, gpu_launches=int(n_launch),
                    clocks=clk, serving=serve, functions=funcs)
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


def serving(pk, seed=1634, n_requests=200, pool_size=8, max_iters=30, load_factor=0.8):
    """Served BA solves: a Poisson stream of requests (2-10 frames x 5k-100k
    LiDAR points, log-uniform, 19-class labels) at load_factor x the measured
    single-stream capacity.  Served form: the request server (continuous
    batching, BF16 labels on the device).  Plain form: one request at a time
    through rkhsba_create + rkhsba_solve with FP32 labels.  Requests are drawn
    from a pool of pool_size generated problems (generation of 200 distinct
    LiDAR problems would dominate the run)."""
    import threading

    import scenes
    specs = scenes.request_stream(seed=seed, n_requests=n_requests)
    pool = []
    for sp in specs[:pool_size]:
        p = scenes.lidar_street_problem(seed=sp["seed"], n_frames=sp["n_frames"],
                                        n_points=sp["n_points"], sem_bf16=1)
        p["params"] = dict(p["params"], max_iters=max_iters)
        pool.append(p)
    rng = np.random.default_rng(seed)
    order = [i % pool_size for i in range(n_requests)]

    def plain_solve(p):
        g = pk.Problem.from_scene(p, sem_bf16=0)
        try:
            return g.solve(p["poses0"])
        finally:
            g.close()

    # single-stream capacity from the plain form on every pool problem
    plain_solve(pool[0])
    svc = []
    for p in pool:
        t0 = time.perf_counter()
        plain_solve(p)
        svc.append(time.perf_counter() - t0)
    mean_svc = sum(svc[order[i]] for i in range(n_requests)) / n_requests
    rate = load_factor / mean_svc
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))

    def pct(x, q):
        return float(np.percentile(np.asarray(x), q))

    # served form
    srv = pk.Server(max_inflight=8)
    lat, done_t = [None] * n_requests, [None] * n_requests
    tickets = [None] * n_requests
    ready = threading.Event()
    fail = []

    def poller():
        ready.wait()
        for i in range(n_requests):
            while tickets[i] is None:
                time.sleep(0.0002)
            r = srv.poll(tickets[i], timeout_ms=-1)
            done_t[i] = time.perf_counter()
            lat[i] = r[1]["latency_ms"]
            if r[1]["state"] != "finished":
                fail.append(r[1])

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    ready.set()
    for i in range(n_requests):
        dt = t0 + arrivals[i] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = srv.submit(pool[order[i]])
    th.join()
    srv.close()
    served_wall = max(done_t) - t0
    served = dict(solves_per_s=n_requests / served_wall, p50_ms=pct(lat, 50), p99_ms=pct(lat, 99),
                  failed=len(fail))

    # plain form: FIFO, one request at a time
    lat2 = []
    t0 = time.perf_counter()
    free_at = t0
    for i in range(n_requests):
        arr = t0 + arrivals[i]
        now = time.perf_counter()
        if now < arr:
            time.sleep(arr - now)
        plain_solve(pool[order[i]])
        fin = time.perf_counter()
        lat2.append(1e3 * (fin - arr))
        free_at = fin
    plain_wall = free_at - t0
    plain = dict(solves_per_s=n_requests / plain_wall, p50_ms=pct(lat2, 50), p99_ms=pct(lat2, 99))

    # capacity: every request queued at once (served) / back to back (plain)
    srv = pk.Server(max_inflight=8)
    t0 = time.perf_counter()
    tk = [srv.submit(pool[order[i]]) for i in range(n_requests)]
    for t in tk:
        srv.poll(t, timeout_ms=-1)
    cap_served = n_requests / (time.perf_counter() - t0)
    srv.close()
    t0 = time.perf_counter()
    for i in range(n_requests):
        plain_solve(pool[order[i]])
    cap_plain = n_requests / (time.perf_counter() - t0)
    served["capacity_solves_per_s"] = cap_served
    plain["capacity_solves_per_s"] = cap_plain
    return dict(metric="served BA solves/s, p50/p99 latency", requests=n_requests, pool=pool_size,
                arrival_rate_per_s=rate, load_factor=load_factor, max_iters=max_iters,
                mean_single_stream_service_ms=1e3 * mean_svc,
                pool_sizes=[[len(p["xyz"]), int(sum(len(x) for x in p["xyz"]))] for p in pool],
                served=served, plain_fp32_single=plain,
                note="solves_per_s and latencies under Poisson arrivals at load_factor x the plain "
                     "single-stream capacity; capacity_solves_per_s with every request queued at once")


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
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="other workloads of the paper's shapes (the driver uses the default)")
    ap.add_argument("--oracle-sample", default=None)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.oracle_sample)))
        return
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

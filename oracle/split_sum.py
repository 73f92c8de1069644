"""The oracle's per-edge sums at full workload size, split over host cores.

TEST INFRASTRUCTURE ONLY (imported by ``tests/`` and by ``bench.py``'s
cpu_baseline leg).  Nothing here adds arithmetic of the method: every sum of
Eq. (inner_product_actual_ba) over the pairs of an edge (a, b) is a sum over
the points y_j of frame b, so ``edge_terms`` of the oracle is evaluated on
consecutive slices of frame b's points (its labels with them) and the slices'
F, E, W, pair counts, b and H are added.  The slices run in a pool of spawned
worker processes (``spawn``: safe after the parent has touched the GPU), each
single-threaded in BLAS, reading the frames from ``.npy`` files that the
parent writes once.

evaluate_split returns what ``oracle.evaluate`` returns for the same edges
(loss, grad, H_blocks, edge_pairs, edge_F, edge_b, n_pairs), in float64.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
import shutil
import tempfile
import time

import numpy as np

from . import rkhs_oracle as O

_cache = {}


def _load(path):
    a = _cache.get(path)
    if a is None:
        a = np.load(path, mmap_mode="r")
        _cache[path] = a
    return a


_ONE_THREAD = {v: "1" for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}


def _init_worker():
    os.environ.update(_ONE_THREAD)


def _slice_terms(task):
    """edge_terms of frame a against points s:e of frame b."""
    (e, fa, fb, s, t, Ta, Tb, params) = task
    xa = np.asarray(_load(fa["xyz"]))
    xb = np.asarray(_load(fb["xyz"])[s:t])
    sa = np.asarray(_load(fa["sem"])) if fa.get("sem") else None
    sb = np.asarray(_load(fb["sem"])[s:t]) if fb.get("sem") else None
    ca = np.asarray(_load(fa["rgb"])) if fa.get("rgb") else None
    cb = np.asarray(_load(fb["rgb"])[s:t]) if fb.get("rgb") else None
    t0 = time.perf_counter()
    r = O.edge_terms(xa, xb, Ta, Tb, sa, sb, ca, cb, params)
    r["seconds"] = time.perf_counter() - t0
    r["edge"] = e
    return r


def _write_frames(problem, frames, tmp):
    out = {}
    sem, rgb = problem.get("sem"), problem.get("rgb")
    for m in frames:
        d = {"xyz": os.path.join(tmp, "xyz%d.npy" % m)}
        np.save(d["xyz"], np.ascontiguousarray(problem["xyz"][m], dtype=np.float64))
        if sem is not None:
            d["sem"] = os.path.join(tmp, "sem%d.npy" % m)
            np.save(d["sem"], np.ascontiguousarray(sem[m], dtype=np.float32))
        if rgb is not None:
            d["rgb"] = os.path.join(tmp, "rgb%d.npy" % m)
            np.save(d["rgb"], np.ascontiguousarray(rgb[m], dtype=np.float32))
        out[m] = d
    return out


def make_pool(workers):
    """A pool of `workers` spawned, single-threaded oracle processes (the BLAS
    thread counts are set in the environment the workers inherit)."""
    os.environ.update(_ONE_THREAD)
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                  initializer=_init_worker)


def evaluate_split(problem, poses, edge_ids, slice_points=4000, workers=None, params=None, pool=None):
    """oracle.evaluate restricted to edge_ids, each edge's frame-b points cut
    into slices of slice_points, the slices evaluated in `workers` spawned
    processes (default: every host core; workers=1 without a pool runs in this
    process) and summed.  `pool` (from make_pool) is used instead of a new one
    when given.  Also returns the wall time, the summed per-slice CPU seconds
    and the worker count."""
    P = O._params(problem["params"])
    if params:
        P.update(params)
    K = len(problem["xyz"])
    edges = np.asarray(problem["edges"]).reshape(-1, 2)
    used = sorted({int(v) for e in edge_ids for v in edges[e]})
    workers = workers or os.cpu_count() or 1
    tmp = tempfile.mkdtemp(prefix="rkhs_oracle_")
    try:
        files = _write_frames(problem, used, tmp)
        tasks = []
        for e in edge_ids:
            a, b = (int(v) for v in edges[e])
            nb = len(problem["xyz"][b])
            for s in range(0, max(nb, 1), slice_points):
                tasks.append((int(e), files[a], files[b], s, min(s + slice_points, nb),
                              np.asarray(poses[a], np.float64), np.asarray(poses[b], np.float64), P))
        t0 = time.perf_counter()
        if pool is not None:
            workers = pool._max_workers
            parts = list(pool.map(_slice_terms, tasks))
        elif workers == 1:
            parts = [_slice_terms(t) for t in tasks]
        else:
            with make_pool(workers) as ex:
                parts = list(ex.map(_slice_terms, tasks))
        wall = time.perf_counter() - t0
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    acc = {int(e): dict(F=0.0, E=0.0, W=0.0, n_pairs=0, b=np.zeros(12), H=np.zeros((12, 12)))
           for e in edge_ids}
    cpu = 0.0
    for r in parts:
        t = acc[r["edge"]]
        for k in ("F", "E", "W"):
            t[k] += r[k]
        t["n_pairs"] += r["n_pairs"]
        t["b"] += r["b"]
        t["H"] += r["H"]
        cpu += r["seconds"]
    F = 0.0
    b = np.zeros(6 * K)
    H = np.zeros((6 * K, 6 * K))
    for e in edge_ids:
        a, bb = (int(v) for v in edges[e])
        t = acc[int(e)]
        idx = np.r_[6 * a:6 * a + 6, 6 * bb:6 * bb + 6]
        F += t["F"]
        b[idx] += t["b"]
        H[np.ix_(idx, idx)] += t["H"]
    scale = P["sigma"] ** 2 / P["ell"] ** 2
    return dict(loss=-F, F=F, grad=scale * b, b=b, H=H,
                H_blocks=np.array([acc[int(e)]["H"] for e in edge_ids]).reshape(-1, 12, 12),
                edge_pairs=np.array([acc[int(e)]["n_pairs"] for e in edge_ids], dtype=np.int64),
                edge_F=np.array([acc[int(e)]["F"] for e in edge_ids]),
                edge_b=np.array([acc[int(e)]["b"] for e in edge_ids]).reshape(-1, 12),
                n_pairs=int(sum(acc[int(e)]["n_pairs"] for e in edge_ids)),
                wall_s=wall, cpu_s=cpu, workers=workers)

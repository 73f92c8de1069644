"""Thin ctypes binding of librkhsba.so (argument marshalling only).

The functions carry the names of the C ABI in include/rkhsba.h; ``Problem``
wraps one context.  Every computation happens in the CUDA library; when the
library cannot be loaded the import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT, EBUSY = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ETIMEOUT",
                6: "EBUSY"}

EXPORTS = [
    "rkhsba_create", "rkhsba_create_device", "rkhsba_destroy", "rkhsba_eval", "rkhsba_solve",
    "rkhsba_set_poses_device", "rkhsba_rebuild", "rkhsba_iterate", "rkhsba_get_state",
    "rkhsba_edge_pairs", "rkhsba_info", "rkhsba_last_error", "rkhsba_launch_count",
    "rkhsba_profile", "rkhsba_server_create", "rkhsba_server_destroy", "rkhsba_submit",
    "rkhsba_poll", "rkhsba_cancel", "rkhsba_server_stats", "rkhsba_inner_products",
    "rkhsba_rotation_search", "rkhsba_solve_ell_decay", "rkhsba_eval_static",
    "rkhsba_selftest_lookback_timeout", "rkhsba_set_tuning", "rkhsba_get_tuning", "rkhsba_autotune",
]


class RkhsbaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Params(C.Structure):
    _fields_ = [("ell", C.c_double), ("cutoff_mult", C.c_double), ("sigma", C.c_double),
                ("ell_color", C.c_double), ("sem_dim", C.c_int32), ("sem_bf16", C.c_int32),
                ("max_iters", C.c_int32), ("top_k", C.c_int32), ("lambda0", C.c_double),
                ("tol_step", C.c_double), ("tol_rel_f", C.c_double), ("sem_min", C.c_double),
                ("cell_scale", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("final_loss", C.c_double),
                ("lam", C.c_double), ("pair_terms", C.c_int64)]


class ServerConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("iters_per_issue", C.c_int32),
                ("memory_budget", C.c_int64), ("request_timeout_ms", C.c_double),
                ("mode", C.c_int32), ("autotune", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("cell_scale", C.c_double), ("unit_queries", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("ms", C.c_double)]


class RequestInfo(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("solve", SolveInfo),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double), ("device_bytes", C.c_int64)]


class EllSchedule(C.Structure):
    _fields_ = [("decay", C.c_double), ("ell_min", C.c_double), ("max_outer", C.c_int32),
                ("reserved", C.c_int32)]


class EllInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("status", C.c_int32), ("ell_final", C.c_double),
                ("final_loss", C.c_double), ("iters", C.c_int64), ("pair_terms", C.c_int64)]


REQUEST_STATES = {0: "queued", 1: "running", 2: "finished", 3: "failed", 4: "cancelled"}


_lib = None
P = C.POINTER


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load librkhsba.so (building it in-tree first when absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("librkhsba.so is missing; run paper_2403_01254_gb300._build.build()")
    lib = C.CDLL(_build.LIB)
    vp = C.c_void_p
    sig = {
        "rkhsba_create": [P(vp), C.c_int32, P(C.c_int64), P(C.c_double), P(C.c_float), P(C.c_float),
                          C.c_int32, P(C.c_int32), P(Params), vp],
        "rkhsba_create_device": [P(vp), C.c_int32, P(C.c_int64), vp, vp, vp, C.c_int32, P(C.c_int32),
                                 P(Params), vp],
        "rkhsba_destroy": [vp],
        "rkhsba_eval": [vp, P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                        P(C.c_int64)],
        "rkhsba_solve": [vp, P(C.c_double), P(SolveInfo)],
        "rkhsba_set_poses_device": [vp, vp],
        "rkhsba_rebuild": [vp],
        "rkhsba_iterate": [vp, C.c_int32],
        "rkhsba_get_state": [vp, P(C.c_double), P(SolveInfo)],
        "rkhsba_edge_pairs": [vp, P(C.c_double), C.c_int32, C.c_int64, P(C.c_int32), P(C.c_int32),
                              P(C.c_int64)],
        "rkhsba_info": [vp, P(C.c_int32), P(C.c_int32), P(C.c_int64), P(C.c_int64)],
        "rkhsba_last_error": [vp],
        "rkhsba_launch_count": [],
        "rkhsba_profile": [vp, C.c_int32, P(C.c_double), P(C.c_int64)],
        "rkhsba_server_create": [P(vp), P(ServerConfig)],
        "rkhsba_server_destroy": [vp],
        "rkhsba_submit": [vp, C.c_int32, P(C.c_int64), P(C.c_double), P(C.c_float), P(C.c_float),
                          C.c_int32, P(C.c_int32), P(Params), P(C.c_double), P(C.c_int64)],
        "rkhsba_poll": [vp, C.c_int64, C.c_int32, P(C.c_double), P(RequestInfo)],
        "rkhsba_cancel": [vp, C.c_int64],
        "rkhsba_server_stats": [vp, P(C.c_int64), P(C.c_int64), P(C.c_int64), P(C.c_int64)],
        "rkhsba_inner_products": [vp, P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double),
                                  P(C.c_double), P(C.c_double)],
        "rkhsba_rotation_search": [vp, C.c_int32, C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double),
                                   P(C.c_double), P(C.c_int32)],
        "rkhsba_solve_ell_decay": [vp, P(EllSchedule), P(C.c_double), P(C.c_double), P(C.c_double),
                                   P(EllInfo)],
        "rkhsba_selftest_lookback_timeout": [C.c_int32, P(C.c_int32)],
        "rkhsba_set_tuning": [vp, C.c_int32, C.c_int32],
        "rkhsba_get_tuning": [vp, P(Tuning)],
        "rkhsba_autotune": [C.c_int32, P(C.c_int64), vp, vp, vp, C.c_int32, P(C.c_int32), P(Params), C.c_int32,
                            P(C.c_double), vp, C.c_int32, P(Tuning), P(Tuning), C.c_int32, P(C.c_int32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.rkhsba_destroy.restype = None
    lib.rkhsba_server_destroy.restype = None
    lib.rkhsba_last_error.restype = C.c_char_p
    lib.rkhsba_launch_count.restype = C.c_int64
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(P(ctype)) if a is not None else None


def _check(status, ctx=None):
    if status != OK:
        msg = load().rkhsba_last_error(ctx)
        raise RkhsbaError(status, msg.decode() if msg else "")
    return status


def make_params(ell, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_dim=0, sem_bf16=0, max_iters=100,
                lambda0=1e-4, tol_step=1e-10, tol_rel_f=1e-12, top_k=0, sem_min=0.0, cell_scale=1.0):
    return Params(float(ell), float(cutoff_mult), float(sigma), float(ell_color), int(sem_dim),
                  int(bool(sem_bf16)), int(max_iters), int(top_k), float(lambda0), float(tol_step),
                  float(tol_rel_f), float(sem_min), float(cell_scale))


# ---------------------------------------------------------------- C-ABI ----
def rkhsba_create(xyz_list, sem_list, rgb_list, edges, params, stream=None):
    """Host arrays -> context handle (int).  xyz_list: K arrays [N_m, 3]."""
    lib = load()
    n = np.array([len(x) for x in xyz_list], dtype=np.int64)
    xyz = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1, 3)
                                               for x in xyz_list]) if len(xyz_list) else
                               np.zeros((0, 3)), dtype=np.float64)
    sem = None
    if sem_list is not None:
        dim = params.sem_dim
        sem = np.ascontiguousarray(np.concatenate([np.asarray(s, np.float32).reshape(len(x), dim)
                                                   for s, x in zip(sem_list, xyz_list)]),
                                   dtype=np.float32)
    rgb = None
    if rgb_list is not None:
        rgb = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float32).reshape(-1, 3)
                                                   for c in rgb_list]), dtype=np.float32)
    e = np.ascontiguousarray(np.asarray(edges, np.int32).reshape(-1))
    h = C.c_void_p()
    _check(lib.rkhsba_create(C.byref(h), len(xyz_list), _ptr(n, C.c_int64), _ptr(xyz, C.c_double),
                             _ptr(sem, C.c_float), _ptr(rgb, C.c_float), len(e) // 2,
                             _ptr(e, C.c_int32), C.byref(params), stream))
    return h.value


def rkhsba_create_flat(n_points, xyz, sem, rgb, edges, params, stream=None):
    """Host arrays already laid out as the C ABI wants them (no copy):
    xyz float64 [N, 3], sem float32 [N, D] or None, rgb float32 [N, 3] or None."""
    lib = load()
    n = np.ascontiguousarray(n_points, dtype=np.int64)
    for a, dt in ((xyz, np.float64), (sem, np.float32), (rgb, np.float32)):
        if a is not None and (a.dtype != dt or not a.flags.c_contiguous):
            raise ValueError("rkhsba_create_flat wants C-contiguous %s arrays" % dt.__name__)
    e = np.ascontiguousarray(np.asarray(edges, np.int32).reshape(-1))
    h = C.c_void_p()
    _check(lib.rkhsba_create(C.byref(h), len(n), _ptr(n, C.c_int64), _ptr(xyz, C.c_double),
                             _ptr(sem, C.c_float), _ptr(rgb, C.c_float), len(e) // 2,
                             _ptr(e, C.c_int32), C.byref(params), stream))
    return h.value


def rkhsba_create_device(n_points, d_xyz, d_sem, d_rgb, edges, params, stream=None):
    """Device pointers (ints) -> context handle."""
    lib = load()
    n = np.ascontiguousarray(n_points, dtype=np.int64)
    e = np.ascontiguousarray(np.asarray(edges, np.int32).reshape(-1))
    h = C.c_void_p()
    _check(lib.rkhsba_create_device(C.byref(h), len(n), _ptr(n, C.c_int64), d_xyz, d_sem, d_rgb,
                                    len(e) // 2, _ptr(e, C.c_int32), C.byref(params), stream))
    return h.value


def rkhsba_destroy(ctx):
    load().rkhsba_destroy(ctx)


def rkhsba_eval(ctx, poses, K, E, want_H=True, want_blocks=False):
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16)
    loss = np.zeros(1)
    grad = np.zeros(6 * K)
    H = np.zeros((6 * K, 6 * K)) if want_H else None
    blocks = np.zeros((E, 12, 12)) if want_blocks else None
    pairs = np.zeros(E, dtype=np.int64)
    _check(load().rkhsba_eval(ctx, _ptr(poses, C.c_double), _ptr(loss, C.c_double),
                              _ptr(grad, C.c_double), _ptr(H, C.c_double), _ptr(blocks, C.c_double),
                              _ptr(pairs, C.c_int64)), ctx)
    return dict(loss=float(loss[0]), grad=grad, H=H, H_blocks=blocks, edge_pairs=pairs,
                n_pairs=int(pairs.sum()))


def rkhsba_solve(ctx, poses, K):
    T = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16).copy()
    info = SolveInfo()
    st = load().rkhsba_solve(ctx, _ptr(T, C.c_double), C.byref(info))
    if st not in (OK, ENOTCONV):
        _check(st, ctx)
    return T.reshape(K, 4, 4), dict(iters=info.iters, status=STATUS_NAMES[info.status],
                                    final_loss=info.final_loss, lam=info.lam,
                                    pair_terms=int(info.pair_terms))


def rkhsba_set_poses_device(ctx, d_poses):
    _check(load().rkhsba_set_poses_device(ctx, d_poses), ctx)


def rkhsba_rebuild(ctx):
    _check(load().rkhsba_rebuild(ctx), ctx)


def rkhsba_iterate(ctx, n):
    _check(load().rkhsba_iterate(ctx, int(n)), ctx)


def rkhsba_get_state(ctx, K):
    T = np.zeros(K * 16)
    info = SolveInfo()
    _check(load().rkhsba_get_state(ctx, _ptr(T, C.c_double), C.byref(info)), ctx)
    return T.reshape(K, 4, 4), dict(iters=info.iters, status=STATUS_NAMES[info.status],
                                    final_loss=info.final_loss, lam=info.lam,
                                    pair_terms=int(info.pair_terms))


def rkhsba_edge_pairs(ctx, poses, K, edge, capacity):
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16)
    i = np.zeros(max(capacity, 1), np.int32)
    j = np.zeros(max(capacity, 1), np.int32)
    n = C.c_int64()
    _check(load().rkhsba_edge_pairs(ctx, _ptr(poses, C.c_double), int(edge), int(capacity),
                                    _ptr(i, C.c_int32), _ptr(j, C.c_int32), C.byref(n)), ctx)
    m = min(n.value, capacity)
    return i[:m].copy(), j[:m].copy(), n.value


def rkhsba_info(ctx):
    k, e, n, b = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
    _check(load().rkhsba_info(ctx, C.byref(k), C.byref(e), C.byref(n), C.byref(b)), ctx)
    return dict(n_frames=k.value, n_edges=e.value, n_points=n.value, device_bytes=b.value)


PHASES = ("grid", "bin", "pairs", "assemble", "solve")


def rkhsba_profile(ctx, enable, read=False):
    """Start (enable=1) / stop (0) phase timing; with read=True return
    {phase: (ms, launches)} of what was recorded (synchronises)."""
    ms = np.zeros(5) if read else None
    n = np.zeros(5, np.int64) if read else None
    _check(load().rkhsba_profile(ctx, int(enable), _ptr(ms, C.c_double), _ptr(n, C.c_int64)), ctx)
    if read:
        return {p: (float(ms[k]), int(n[k])) for k, p in enumerate(PHASES)}
    return None


def rkhsba_inner_products(ctx, poses, K, E):
    """Self terms <f_m,f_m> [K], per-edge <f_a,f_b>, |f_a-f_b|^2 and cosine [E],
    and d(sum dist)/d ell (Eq. dist_rkhs)."""
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16)
    self_ip, cross, dist, cos, dD = np.zeros(K), np.zeros(E), np.zeros(E), np.zeros(E), np.zeros(1)
    _check(load().rkhsba_inner_products(ctx, _ptr(poses, C.c_double), _ptr(self_ip, C.c_double),
                                        _ptr(cross, C.c_double), _ptr(dist, C.c_double),
                                        _ptr(cos, C.c_double), _ptr(dD, C.c_double)), ctx)
    return dict(self=self_ip, cross=cross, dist=dist, cos=cos, dD_dell=float(dD[0]))


def rkhsba_rotation_search(ctx, a, b, poses, K):
    """Cosines of the 60 icosahedral candidates of frame b against frame a,
    the rotations R_k [60,3,3], the best candidate's pose of b and its index."""
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16)
    cos, rot, best_pose, best = np.zeros(60), np.zeros(540), np.zeros(16), C.c_int32()
    _check(load().rkhsba_rotation_search(ctx, int(a), int(b), _ptr(poses, C.c_double), _ptr(cos, C.c_double),
                                         _ptr(rot, C.c_double), _ptr(best_pose, C.c_double),
                                         C.byref(best)), ctx)
    return dict(cos=cos, rotations=rot.reshape(60, 3, 3), best_pose=best_pose.reshape(4, 4),
                best=best.value)


def rkhsba_solve_ell_decay(ctx, poses, K, decay=0.1, ell_min=0.0, max_outer=10):
    """Lengthscale-decay outer loop around the LM solve (Sec. V-C)."""
    T = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16).copy()
    sched = EllSchedule(float(decay), float(ell_min), int(max_outer), 0)
    ells, dDs, info = np.zeros(max_outer), np.zeros(max_outer), EllInfo()
    _check(load().rkhsba_solve_ell_decay(ctx, C.byref(sched), _ptr(T, C.c_double), _ptr(ells, C.c_double),
                                         _ptr(dDs, C.c_double), C.byref(info)), ctx)
    n = info.levels
    return T.reshape(K, 4, 4), dict(levels=n, ell=ells[:n].copy(), dD_dell=dDs[:n].copy(),
                                    status=STATUS_NAMES[info.status], ell_final=info.ell_final,
                                    final_loss=info.final_loss, iters=int(info.iters),
                                    pair_terms=int(info.pair_terms))


def rkhsba_selftest_lookback_timeout(spin_limit=1000):
    """Make one bounded look-back wait of the radix sort run out (failure
    detection self-test).  Returns (status name, writes_in_bounds)."""
    ok = C.c_int32(0)
    st = load().rkhsba_selftest_lookback_timeout(int(spin_limit), C.byref(ok))
    if st not in (OK, ETIMEOUT):
        _check(st)
    return STATUS_NAMES[st], bool(ok.value)


def _tuning_dict(t):
    return dict(cell_scale=t.cell_scale, unit_queries=t.unit_queries, ctas_per_sm=t.ctas_per_sm, ms=t.ms)


def rkhsba_set_tuning(ctx, unit_queries=32, ctas_per_sm=0):
    _check(load().rkhsba_set_tuning(ctx, int(unit_queries), int(ctas_per_sm)), ctx)


def rkhsba_get_tuning(ctx):
    t = Tuning()
    _check(load().rkhsba_get_tuning(ctx, C.byref(t)), ctx)
    return _tuning_dict(t)


def rkhsba_autotune(n_points, xyz, sem, rgb, edges, params, poses, stream=None, reps=2, on_device=False):
    """Time the evaluation under every candidate (cell_scale, unit_queries,
    ctas_per_sm); returns (best, table) as dicts.  xyz / sem / rgb: flat host
    arrays (float64 [N,3], float32 [N,D], float32 [N,3] or None), or device
    pointers (ints) with on_device=True."""
    lib = load()
    n = np.ascontiguousarray(n_points, dtype=np.int64)
    K = len(n)
    e = np.ascontiguousarray(np.asarray(edges, np.int32).reshape(-1))
    T = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16)
    if on_device:
        px, ps, pr = xyz, sem, rgb
    else:
        px, ps, pr = (None if a is None else a.ctypes.data for a in (xyz, sem, rgb))
    best = Tuning()
    table = (Tuning * 32)()
    nt = C.c_int32()
    _check(lib.rkhsba_autotune(K, _ptr(n, C.c_int64), px, ps, pr, len(e) // 2, _ptr(e, C.c_int32),
                               C.byref(params), int(bool(on_device)), _ptr(T, C.c_double), stream, int(reps),
                               C.byref(best), table, 32, C.byref(nt)))
    return _tuning_dict(best), [_tuning_dict(table[i]) for i in range(min(nt.value, 32))]


def rkhsba_launch_count():
    return int(load().rkhsba_launch_count())


# ------------------------------------------------------------- wrapper -----
class Problem:
    """One RKHS-BA problem resident on the GPU (a C-ABI context)."""

    def __init__(self, xyz, sem=None, rgb=None, edges=None, ell=0.1, cutoff_mult=3.0, sigma=1.0,
                 ell_color=0.0, sem_bf16=False, max_iters=100, lambda0=1e-4, tol_step=1e-10,
                 tol_rel_f=1e-12, top_k=0, sem_min=0.0, cell_scale=1.0, stream=None):
        self.K = len(xyz)
        self.edges = np.asarray(edges, np.int32).reshape(-1, 2)
        self.E = len(self.edges)
        sem_dim = 0 if sem is None else int(np.asarray(sem[0]).shape[-1])
        self.params = make_params(ell, cutoff_mult, sigma, ell_color, sem_dim, sem_bf16, max_iters,
                                  lambda0, tol_step, tol_rel_f, top_k, sem_min, cell_scale)
        self.ctx = rkhsba_create(xyz, sem, rgb, self.edges, self.params, stream)

    @classmethod
    def from_scene(cls, prob, **over):
        p = dict(prob["params"])
        p.update(over)
        keep = {k: p[k] for k in ("ell", "cutoff_mult", "sigma", "ell_color", "sem_bf16", "max_iters",
                                  "lambda0", "tol_step", "tol_rel_f", "top_k", "sem_min", "cell_scale") if k in p}
        return cls(prob["xyz"], prob.get("sem"), prob.get("rgb"), prob["edges"], **keep)

    def eval(self, poses, want_H=True, want_blocks=False):
        return rkhsba_eval(self.ctx, poses, self.K, self.E, want_H, want_blocks)

    def solve(self, poses0):
        return rkhsba_solve(self.ctx, poses0, self.K)

    def edge_pairs(self, poses, edge, capacity=1 << 24):
        return rkhsba_edge_pairs(self.ctx, poses, self.K, edge, capacity)

    def inner_products(self, poses):
        return rkhsba_inner_products(self.ctx, poses, self.K, self.E)

    def rotation_search(self, a, b, poses):
        return rkhsba_rotation_search(self.ctx, a, b, poses, self.K)

    def solve_ell_decay(self, poses0, decay=0.1, ell_min=0.0, max_outer=10):
        return rkhsba_solve_ell_decay(self.ctx, poses0, self.K, decay, ell_min, max_outer)

    def info(self):
        return rkhsba_info(self.ctx)

    def set_tuning(self, unit_queries=32, ctas_per_sm=0):
        rkhsba_set_tuning(self.ctx, unit_queries, ctas_per_sm)

    def tuning(self):
        return rkhsba_get_tuning(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            rkhsba_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rkhsba_eval_static(n_points, d_xyz, d_sem, d_rgb, edges, params, poses, stream=None):
    """Evaluation without device allocation (rkhsba_eval_static in the C ABI).

    For callers that cannot allocate device memory: the library runs the
    evaluation in a fixed scratch array of its own.  d_xyz / d_sem / d_rgb are
    device pointers (ints, or None); results come back as host arrays.
    """
    lib = load()
    f = lib.rkhsba_eval_static
    if f.argtypes is None:
        f.argtypes = [C.c_int32, P(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                      P(C.c_int32), P(Params), P(C.c_double), P(C.c_double), P(C.c_double),
                      P(C.c_double), C.c_void_p]
        f.restype = C.c_int
    n = np.ascontiguousarray(n_points, dtype=np.int64)
    K = len(n)
    e = np.ascontiguousarray(np.asarray(edges, np.int32).reshape(-1))
    T = np.ascontiguousarray(poses, dtype=np.float64).reshape(K * 16)
    loss = np.zeros(1)
    grad = np.zeros(6 * K)
    H = np.zeros((6 * K, 6 * K))
    _check(f(K, _ptr(n, C.c_int64), d_xyz, d_sem, d_rgb, len(e) // 2, _ptr(e, C.c_int32),
             C.byref(params), _ptr(T, C.c_double), _ptr(loss, C.c_double), _ptr(grad, C.c_double),
             _ptr(H, C.c_double), stream))
    return dict(loss=float(loss[0]), grad=grad, H=H)


# ------------------------------------------------------------- server ------
class Server:
    """Continuous-batching request server (rkhsba_server_* in the C ABI)."""

    MODES = {"batched": 0, "per_request": 1}

    def __init__(self, max_inflight=8, iters_per_issue=4, memory_budget=0, request_timeout_ms=0.0,
                 mode="batched", autotune=False):
        lib = load()
        cfg = ServerConfig(int(max_inflight), int(iters_per_issue), int(memory_budget),
                           float(request_timeout_ms), self.MODES[mode], int(bool(autotune)))
        h = C.c_void_p()
        _check(lib.rkhsba_server_create(C.byref(h), C.byref(cfg)))
        self.h = h.value
        self.K = {}

    def submit(self, prob, poses0=None, **over):
        """Queue a problem dict (as produced by ``scenes``); returns a ticket."""
        lib = load()
        p = dict(prob["params"])
        p.update(over)
        K = len(prob["xyz"])
        sem = prob.get("sem")
        sem_dim = 0 if sem is None else int(np.asarray(sem[0]).shape[-1])
        params = make_params(p["ell"], p.get("cutoff_mult", 3.0), p.get("sigma", 1.0),
                             p.get("ell_color", 0.0), sem_dim, p.get("sem_bf16", 0),
                             p.get("max_iters", 100), p.get("lambda0", 1e-4),
                             p.get("tol_step", 1e-10), p.get("tol_rel_f", 1e-12), p.get("top_k", 0),
                             p.get("sem_min", 0.0), p.get("cell_scale", 1.0))
        n = np.array([len(x) for x in prob["xyz"]], np.int64)
        xyz = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1, 3)
                                                   for x in prob["xyz"]]))
        semf = None
        if sem is not None:
            semf = np.ascontiguousarray(np.concatenate([np.asarray(s_, np.float32).reshape(len(x), sem_dim)
                                                        for s_, x in zip(sem, prob["xyz"])]))
        rgb = prob.get("rgb")
        rgbf = None
        if rgb is not None and p.get("ell_color", 0.0) > 0:
            rgbf = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float32).reshape(-1, 3)
                                                        for c in rgb]))
        e = np.ascontiguousarray(np.asarray(prob["edges"], np.int32).reshape(-1))
        T0 = np.ascontiguousarray(prob["poses0"] if poses0 is None else poses0,
                                  dtype=np.float64).reshape(K * 16)
        t = C.c_int64()
        _check(lib.rkhsba_submit(self.h, K, _ptr(n, C.c_int64), _ptr(xyz, C.c_double),
                                 _ptr(semf, C.c_float), _ptr(rgbf, C.c_float), len(e) // 2,
                                 _ptr(e, C.c_int32), C.byref(params), _ptr(T0, C.c_double),
                                 C.byref(t)))
        self.K[t.value] = K
        return t.value

    def poll(self, ticket, timeout_ms=-1):
        """(poses or None, info) once the request ended, None while it runs."""
        K = self.K[ticket]
        T = np.zeros(K * 16)
        info = RequestInfo()
        st = load().rkhsba_poll(self.h, int(ticket), int(timeout_ms), _ptr(T, C.c_double),
                                C.byref(info))
        if st == EBUSY:
            return None
        _check(st)
        del self.K[ticket]
        d = dict(state=REQUEST_STATES[info.state], status=STATUS_NAMES.get(info.status, info.status),
                 iters=info.solve.iters, final_loss=info.solve.final_loss,
                 pair_terms=int(info.solve.pair_terms), queue_ms=info.queue_ms,
                 latency_ms=info.latency_ms, device_bytes=int(info.device_bytes))
        return (T.reshape(K, 4, 4) if info.state == 2 else None), d

    def cancel(self, ticket):
        _check(load().rkhsba_cancel(self.h, int(ticket)))

    def stats(self):
        q, r, f, b = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().rkhsba_server_stats(self.h, C.byref(q), C.byref(r), C.byref(f), C.byref(b)))
        return dict(queued=q.value, running=r.value, finished=f.value, device_bytes=b.value)

    def close(self):
        if getattr(self, "h", None):
            load().rkhsba_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rkhsba_server_create(max_inflight=8, iters_per_issue=4, memory_budget=0, request_timeout_ms=0.0,
                         mode="batched", autotune=False):
    return Server(max_inflight, iters_per_issue, memory_budget, request_timeout_ms, mode, autotune)


def rkhsba_server_destroy(server):
    server.close()


def rkhsba_submit(server, prob, poses0=None, **over):
    return server.submit(prob, poses0, **over)


def rkhsba_poll(server, ticket, timeout_ms=-1):
    return server.poll(ticket, timeout_ms)


def rkhsba_cancel(server, ticket):
    server.cancel(ticket)


def rkhsba_server_stats(server):
    return server.stats()

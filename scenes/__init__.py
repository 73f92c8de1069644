"""Seeded synthetic RKHS-BA problems (input generation only).

This module is shared by the tests, ``bench.py`` and the oracle checks.  It
holds no arithmetic of the method itself: no kernel weights, no gradients,
no SE(3) exponential or logarithm.  Rotations are built from unit
quaternions, LiDAR returns by casting rays against a few analytic
primitives, and labels by sampling one-hot or Dirichlet class vectors.

The shapes mirror the paper's workloads (Sec. VI): RGB-D-like frames of a
few thousand points with <= 10 classes, LiDAR frames with semantic class
distributions, multi-view registration from random rotations/translations,
sliding windows on a trajectory and a global mapping batch with loop
closures.  No dataset content is reproduced; every scene is procedural.

A problem is a plain dict:
    xyz      list of float64 [N_m, 3] frame-local points
    sem      list of float32 [N_m, D] label vectors, or None
    rgb      list of float32 [N_m, 3] colours in [0, 1], or None
    edges    int32 [E, 2], a < b, every unordered pair at most once
    poses_gt float64 [K, 4, 4] frame-to-world ground truth
    poses0   float64 [K, 4, 4] initial guess (frame 0 equals ground truth)
    params   dict(ell, cutoff_mult, sigma, ell_color, sem_bf16)
    name     short workload name
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rot_from_axis_angle", "random_rotation_deg", "make_pose", "random_pose",
    "perturb", "to_local", "plane_sphere_problem", "lidar_street_problem",
    "window_problem", "mapping_problem", "request_stream", "tiny_problem",
    "config_problem",
]


# --------------------------------------------------------------------------
# rigid poses (quaternion based; independent of any exp/log map)
# --------------------------------------------------------------------------
def rot_from_axis_angle(axis, angle):
    """Rotation matrix of ``angle`` radians about ``axis`` via a unit quaternion."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    w = math.cos(angle / 2.0)
    x, y, z = axis * math.sin(angle / 2.0)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def random_rotation_deg(rng, angle_deg):
    axis = rng.normal(size=3)
    return rot_from_axis_angle(axis, math.radians(angle_deg))


def make_pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def random_pose(rng, angle_deg, trans):
    """Pose with rotation of exactly ``angle_deg`` about a random axis and a
    translation of length ``trans`` in a random direction."""
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    return make_pose(random_rotation_deg(rng, angle_deg), trans * u)


def perturb(rng, T, max_deg, max_trans):
    """Right-multiply ``T`` by a random pose of angle <= max_deg, |t| <= max_trans."""
    P = random_pose(rng, rng.uniform(0.0, max_deg), rng.uniform(0.0, max_trans))
    return T @ P


def to_local(xyz_world, T):
    """Express world points in the frame whose frame-to-world pose is T."""
    R, t = T[:3, :3], T[:3, 3]
    return (xyz_world - t) @ R


def _yaw_pose(x, y, z, yaw):
    c, s = math.cos(yaw), math.sin(yaw)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return make_pose(R, np.array([x, y, z]))


# --------------------------------------------------------------------------
# input storage formats
# --------------------------------------------------------------------------
def round_to_bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even); returned as
    float32 so that a later float32 -> bfloat16 conversion is exact."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def round_to_f32(a):
    """Points stored as float32 upstream (e.g. a sensor driver)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# labels
# --------------------------------------------------------------------------
def one_hot(labels, n_classes):
    out = np.zeros((len(labels), n_classes), dtype=np.float32)
    out[np.arange(len(labels)), labels] = 1.0
    return out


def dirichlet_labels(rng, labels, n_classes, alpha=0.3, peak=10.0):
    """Class-probability vectors: Dirichlet(alpha * 1 + peak * e_class)."""
    a = np.full((len(labels), n_classes), alpha)
    a[np.arange(len(labels)), labels % n_classes] += peak
    g = rng.gamma(a)
    return (g / g.sum(axis=1, keepdims=True)).astype(np.float32)


# --------------------------------------------------------------------------
# config 1: three planes and a sphere in a 10 m cube (RGB-D-like)
# --------------------------------------------------------------------------
_PS_COLORS = np.array([[0.55, 0.45, 0.35], [0.80, 0.80, 0.75],
                       [0.30, 0.45, 0.70], [0.85, 0.20, 0.15]])


def _sample_planes_sphere(rng, n, noise):
    areas = np.array([100.0, 100.0, 100.0, 4.0 * math.pi * 1.5 ** 2])
    prim = rng.choice(4, size=n, p=areas / areas.sum())
    pts = np.empty((n, 3))
    u = rng.uniform(0.0, 10.0, size=(n, 2))
    m = prim == 0  # floor z = 0
    pts[m] = np.c_[u[m, 0], u[m, 1], np.zeros(m.sum())]
    m = prim == 1  # wall x = 0
    pts[m] = np.c_[np.zeros(m.sum()), u[m, 0], u[m, 1]]
    m = prim == 2  # wall y = 0
    pts[m] = np.c_[u[m, 0], np.zeros(m.sum()), u[m, 1]]
    m = prim == 3  # sphere centre (5, 5, 3), radius 1.5
    v = rng.normal(size=(m.sum(), 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts[m] = np.array([5.0, 5.0, 3.0]) + 1.5 * v
    pts += rng.normal(scale=noise, size=pts.shape)
    rgb = np.clip(_PS_COLORS[prim] + rng.normal(scale=0.02, size=(n, 3)), 0.0, 1.0)
    return pts, prim, rgb.astype(np.float32)


def plane_sphere_problem(seed=1334, n=2000, noise=0.01, angle_deg=10.0, trans=0.3,
                         ell=0.1, ell_color=0.1, n_classes=5, same_points=False):
    """Two RGB-D-like frames of ``n`` points; frame 1 under a random pose."""
    rng = np.random.default_rng(seed)
    p0, l0, c0 = _sample_planes_sphere(rng, n, noise)
    if same_points:
        p1, l1, c1 = p0.copy(), l0.copy(), c0.copy()
    else:
        p1, l1, c1 = _sample_planes_sphere(rng, n, noise)
    T1 = random_pose(rng, angle_deg, trans)
    poses_gt = np.stack([np.eye(4), T1])
    return dict(
        name="plane_sphere_2x%d" % n,
        xyz=[p0, to_local(p1, T1)],
        sem=[one_hot(l0, n_classes), one_hot(l1, n_classes)],
        rgb=[c0, c1],
        edges=np.array([[0, 1]], dtype=np.int32),
        poses_gt=poses_gt,
        poses0=np.stack([np.eye(4), np.eye(4)]),
        params=dict(ell=ell, cutoff_mult=3.0, sigma=1.0, ell_color=ell_color, sem_bf16=0),
    )


# --------------------------------------------------------------------------
# two scans of one asymmetric object under a large rotation (global
# initialisation protocol of Sec. VI-A: 90 / 180 degrees about a random axis,
# translation of length 0.5, normal-direction noise with outliers, cropping)
# --------------------------------------------------------------------------
def _sample_object(rng, n):
    """Surface points, unit normals and part index of a body (ellipsoid), a
    head (cube) and a tail (cylinder); the union has no symmetry."""
    areas = np.array([0.86, 0.375, 0.226])
    prim = rng.choice(3, size=n, p=areas / areas.sum())
    pts = np.empty((n, 3))
    nrm = np.empty((n, 3))
    m = prim == 0                                     # ellipsoid, radii (0.4, 0.25, 0.15)
    rad = np.array([0.4, 0.25, 0.15])
    v = rng.normal(size=(m.sum(), 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts[m] = v * rad
    g = v / rad
    nrm[m] = g / np.linalg.norm(g, axis=1, keepdims=True)
    m = prim == 1                                     # cube of side 0.25 at (0.45, 0.2, 0.12)
    k = int(m.sum())
    face = rng.integers(0, 6, size=k)
    uv = rng.uniform(-0.125, 0.125, size=(k, 2))
    ax = face // 2
    sgn = np.where(face % 2 == 0, 1.0, -1.0)
    q = np.zeros((k, 3))
    e = np.zeros((k, 3))
    for a in range(3):
        sel = ax == a
        o = [b for b in range(3) if b != a]
        q[sel, a] = 0.125 * sgn[sel]
        q[sel, o[0]] = uv[sel, 0]
        q[sel, o[1]] = uv[sel, 1]
        e[sel, a] = sgn[sel]
    pts[m] = q + np.array([0.45, 0.2, 0.12])
    nrm[m] = e
    m = prim == 2                                     # cylinder r = 0.06, length 0.6
    k = int(m.sum())
    d = np.array([-1.0, 0.3, 0.5])
    d /= np.linalg.norm(d)
    u1 = np.cross(d, [0.0, 0.0, 1.0])
    u1 /= np.linalg.norm(u1)
    u2 = np.cross(d, u1)
    th = rng.uniform(0, 2 * math.pi, size=k)
    s = rng.uniform(0, 0.6, size=k)
    radial = np.cos(th)[:, None] * u1 + np.sin(th)[:, None] * u2
    pts[m] = np.array([-0.35, 0.0, 0.0]) + s[:, None] * d + 0.06 * radial
    nrm[m] = radial
    return pts, nrm, prim


def _scan(rng, n, outlier_ratio, crop_ratio):
    pts, nrm, prim = _sample_object(rng, n)
    out = rng.uniform(size=n) < outlier_ratio
    off = np.where(out, rng.uniform(-0.1, 0.1, size=n), rng.normal(scale=0.01, size=n))
    pts = pts + off[:, None] * nrm
    if crop_ratio > 0:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        h = pts @ u
        keep = h <= np.quantile(h, 1.0 - crop_ratio)
        pts, prim = pts[keep], prim[keep]
    return pts, prim


def object_pair_problem(seed=1834, angle_deg=90.0, trans=0.5, n=2000, outlier_ratio=0.0, crop_ratio=0.0,
                        ell=0.1, labels=False):
    """Two independent noisy scans of the object; frame 1 under a rotation of
    angle_deg about a random axis and a translation of length trans.  With
    labels, each point carries a Dirichlet class vector peaked at its part
    (body, head, tail): a pose-invariant descriptor standing in for the
    per-point features of the label function."""
    rng = np.random.default_rng(seed)
    p0, l0 = _scan(rng, n, outlier_ratio, crop_ratio)
    p1, l1 = _scan(rng, n, outlier_ratio, crop_ratio)
    T1 = random_pose(rng, angle_deg, trans)
    sem = [dirichlet_labels(rng, l0, 3), dirichlet_labels(rng, l1, 3)] if labels else None
    return dict(
        name="object_pair_%ddeg" % int(round(angle_deg)),
        xyz=[p0, to_local(p1, T1)],
        sem=sem,
        rgb=None,
        edges=np.array([[0, 1]], dtype=np.int32),
        poses_gt=np.stack([np.eye(4), T1]),
        poses0=np.stack([np.eye(4), np.eye(4)]),
        params=dict(ell=ell, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_bf16=0),
    )


# --------------------------------------------------------------------------
# LiDAR street scene (configs 2-5)
# --------------------------------------------------------------------------
def _street_primitives(rng, x_range=(-70.0, 70.0), half_width=8.0):
    """Ground, two facades, poles and parked boxes.  Returns (boxes, poles):
    boxes as [lo(3), hi(3), class]; poles as [x, y, radius, height, class]."""
    x0, x1 = x_range
    boxes = [
        ([x0, half_width, 0.0], [x1, half_width + 2.0, 15.0], 2),      # facade left
        ([x0, -half_width - 2.0, 0.0], [x1, -half_width, 15.0], 3),    # facade right
    ]
    # parked boxes (cars) along both kerbs
    for side in (-1.0, 1.0):
        x = x0 + rng.uniform(0.0, 6.0)
        while x < x1 - 5.0:
            y = side * (half_width - 2.2)
            L, W, H = rng.uniform(3.8, 4.8), rng.uniform(1.7, 1.95), rng.uniform(1.4, 1.7)
            cls = 4 + int(rng.integers(0, 3))
            boxes.append(([x, y - W / 2, 0.0], [x + L, y + W / 2, H], cls))
            x += L + rng.uniform(1.0, 9.0)
    poles = []
    for side in (-1.0, 1.0):
        x = x0 + rng.uniform(0.0, 10.0)
        while x < x1:
            poles.append((x, side * (half_width - 0.8), 0.12, 6.0, 7 + int(rng.integers(0, 2))))
            x += rng.uniform(8.0, 16.0)
    return boxes, poles


def _cast(origins, dirs, boxes, poles, rmin, rmax):
    """Nearest hit distance and class per ray against ground/boxes/poles.
    Rays share one origin per scan; a box or pole farther than rmax from it
    cannot give a hit in range and is skipped (the hit set, its distances and
    classes do not change)."""
    n = len(dirs)
    best = np.full(n, np.inf)
    cls = np.full(n, -1, dtype=np.int64)
    o = origins
    o0 = np.asarray(o[0], dtype=np.float64)
    # ground plane z = 0 (class 0 road)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = -o[:, 2] / dirs[:, 2]
        inv = 1.0 / dirs
    ok = (dirs[:, 2] < 0) & (t > 0) & (t < best)
    best[ok] = t[ok]
    cls[ok] = 0
    # axis-aligned boxes (slab method); fmax/fmin skip the NaN of 0 * inf
    for lo, hi, c in boxes:
        lo = np.asarray(lo)
        hi = np.asarray(hi)
        gap = np.maximum(np.maximum(lo - o0, o0 - hi), 0.0)
        if float(np.sqrt(gap @ gap)) > rmax:
            continue
        with np.errstate(invalid="ignore"):
            t1 = (lo - o0) * inv
            t2 = (hi - o0) * inv
        a = np.minimum(t1, t2)
        b = np.maximum(t1, t2)
        tmin = np.fmax(np.fmax(a[:, 0], a[:, 1]), a[:, 2])
        tmax = np.fmin(np.fmin(b[:, 0], b[:, 1]), b[:, 2])
        ok = (tmax >= tmin) & (tmin > 0) & (tmin < best)
        best[ok] = tmin[ok]
        cls[ok] = c
    # vertical cylinders
    for px, py, r, h, c in poles:
        if math.hypot(o0[0] - px, o0[1] - py) - r > rmax:
            continue
        dx = o0[0] - px
        dy = o0[1] - py
        a = dirs[:, 0] ** 2 + dirs[:, 1] ** 2
        b = 2 * (dx * dirs[:, 0] + dy * dirs[:, 1])
        cc = dx * dx + dy * dy - r * r
        disc = b * b - 4 * a * cc
        ok = disc > 0
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (-b - np.sqrt(np.where(ok, disc, 0.0))) / (2 * a)
        z = o[:, 2] + t * dirs[:, 2]
        ok &= (t > 0) & (t < best) & (z >= 0) & (z <= h)
        best[ok] = t[ok]
        cls[ok] = c
    hit = (best >= rmin) & (best <= rmax)
    return best, cls, hit


def lidar_scan(rng, T_sensor, boxes, poles, n_beams=64, n_az=312, elev=(-25.0, 3.0),
               rmin=1.0, rmax=50.0, noise=0.01):
    """One ring-pattern scan; returns world points and their classes."""
    el = np.radians(np.linspace(elev[0], elev[1], n_beams))
    az = np.radians(np.arange(n_az) * (360.0 / n_az)) + rng.uniform(0, 2 * math.pi / n_az)
    E, A = np.meshgrid(el, az, indexing="ij")
    d_local = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1).reshape(-1, 3)
    R, t = T_sensor[:3, :3], T_sensor[:3, 3]
    dirs = d_local @ R.T
    origins = np.broadcast_to(t, dirs.shape)
    rng_dist, cls, hit = _cast(origins, dirs, boxes, poles, rmin, rmax)
    r = rng_dist[hit] + rng.normal(scale=noise, size=hit.sum())
    pts = origins[hit] + dirs[hit] * r[:, None]
    return pts, cls[hit]


def _lidar_problem(rng, sensor_poses, n_points, boxes, poles, n_classes, noise, outliers,
                   sem_bf16, ell, edges, poses0, name, xyz_f32=False):
    n_az = max(8, int(round(n_points / 64)))
    xyz, sem = [], []
    all_world = []
    for T in sensor_poses:
        pts, cls = lidar_scan(rng, T, boxes, poles, n_az=n_az, noise=noise)
        if outliers > 0:
            n_out = int(round(outliers * len(pts)))
            lo, hi = pts.min(0), pts.max(0)
            out = rng.uniform(lo, hi, size=(n_out, 3))
            idx = rng.choice(len(pts), size=n_out, replace=False)
            pts = pts.copy()
            pts[idx] = out
            cls = cls.copy()
            cls[idx] = rng.integers(0, n_classes, size=n_out)
        all_world.append(pts)
        local = to_local(pts, T)
        xyz.append(round_to_f32(local) if xyz_f32 else local)
        lab = dirichlet_labels(rng, cls, n_classes)
        sem.append(round_to_bf16(lab) if sem_bf16 else lab)
    return dict(
        name=name, xyz=xyz, sem=sem, rgb=None,
        edges=np.asarray(edges, dtype=np.int32).reshape(-1, 2),
        poses_gt=np.stack(sensor_poses), poses0=np.stack(poses0),
        params=dict(ell=ell, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_bf16=sem_bf16),
    )


def all_pairs(K):
    return [(a, b) for a in range(K) for b in range(a + 1, K)]


def lidar_street_problem(seed=1434, n_frames=8, n_points=20000, max_deg=15.0, max_trans=0.5,
                         ell=0.3, n_classes=19, sem_bf16=0, noise=0.01, outliers=0.0,
                         spacing=1.5):
    """Multi-view registration: ``n_frames`` scans along a street, all pairs."""
    rng = np.random.default_rng(seed)
    boxes, poles = _street_primitives(rng)
    gt = [_yaw_pose(spacing * k - spacing * (n_frames - 1) / 2, rng.uniform(-1, 1), 1.7,
                    math.radians(rng.uniform(-5, 5))) for k in range(n_frames)]
    init = [gt[0]] + [perturb(rng, T, max_deg, max_trans) for T in gt[1:]]
    return _lidar_problem(rng, gt, n_points, boxes, poles, n_classes, noise, outliers,
                          sem_bf16, ell, all_pairs(n_frames), init,
                          "lidar_street_%dx%d" % (n_frames, n_points))


def window_problem(seed=1534, window=5, n_points=50000, ell=0.3, n_classes=19,
                   noise=0.02, outliers=0.10, max_deg=2.0, max_trans=0.1):
    """Sliding-window odometry: consecutive poses 1 m apart on a smooth yaw path."""
    rng = np.random.default_rng(seed)
    boxes, poles = _street_primitives(rng)
    yaw, x, y = 0.0, -window / 2.0, 0.0
    gt = []
    for _ in range(window):
        gt.append(_yaw_pose(x, y, 1.7, yaw))
        yaw += math.radians(rng.normal(0.0, 1.5))
        x += math.cos(yaw)
        y += math.sin(yaw)
    init = [gt[0]] + [perturb(rng, T, max_deg, max_trans) for T in gt[1:]]
    return _lidar_problem(rng, gt, n_points, boxes, poles, n_classes, noise, outliers,
                          1, ell, all_pairs(window), init,
                          "window_%dx%d" % (window, n_points), xyz_f32=True)


def mapping_problem(seed=1734, n_frames=64, n_points=100000, lap=16, ell=0.3,
                    n_classes=19, near=7, max_deg=1.0, max_trans=0.05, closure=0.5):
    """Global mapping batch: a loop of ``lap`` m walked at 1 m/frame, edges
    |i-j| <= near plus loop closures between revisiting frames (closer than
    ``closure`` m).  64 frames, lap 16, near 7 give 420 + 96 = 516 edges."""
    rng = np.random.default_rng(seed)
    boxes, poles = _street_primitives(rng)
    radius = lap / (2 * math.pi)
    gt = []
    for k in range(n_frames):
        th = 2 * math.pi * k / lap
        gt.append(_yaw_pose(radius * math.cos(th), radius * math.sin(th), 1.7,
                            th + math.pi / 2))
    edges = []
    for a in range(n_frames):
        for b in range(a + 1, n_frames):
            close = np.linalg.norm(gt[a][:3, 3] - gt[b][:3, 3]) < closure
            if b - a <= near or close:
                edges.append((a, b))
    init = [gt[0]] + [perturb(rng, T, max_deg, max_trans) for T in gt[1:]]
    return _lidar_problem(rng, gt, n_points, boxes, poles, n_classes, 0.02, 0.0,
                          1, ell, edges, init, "mapping_%dx%d" % (n_frames, n_points))


def request_stream(seed=1634, n_requests=200, frames=(2, 10), points=(5000, 100000)):
    """Served stream: per request (arrival_index, problem-spec kwargs).  Problems
    are built lazily by ``lidar_street_problem`` with the returned kwargs."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_requests):
        k = int(rng.integers(frames[0], frames[1] + 1))
        n = int(round(math.exp(rng.uniform(math.log(points[0]), math.log(points[1])))))
        out.append(dict(seed=int(rng.integers(1 << 30)), n_frames=k, n_points=n,
                        sem_bf16=1))
    return out


def tiny_problem(seed=7, n_frames=3, n=60, extent=1.0, ell=0.15, n_classes=4,
                 color=False, max_deg=5.0, max_trans=0.05, edges=None):
    """A few dozen points per frame in a small box; for brute-force checks."""
    rng = np.random.default_rng(seed)
    base = rng.uniform(0, extent, size=(n, 3))
    lab = rng.integers(0, n_classes, size=n)
    gt = [np.eye(4)] + [random_pose(rng, rng.uniform(0, 20), rng.uniform(0, 0.3))
                        for _ in range(n_frames - 1)]
    xyz, sem, rgb = [], [], []
    for T in gt:
        pts = base + rng.normal(scale=0.01, size=base.shape)
        xyz.append(to_local(pts, T))
        sem.append(dirichlet_labels(rng, lab, n_classes, alpha=0.5, peak=4.0))
        rgb.append(rng.uniform(0, 1, size=(n, 3)).astype(np.float32))
    init = [gt[0]] + [perturb(rng, T, max_deg, max_trans) for T in gt[1:]]
    return dict(
        name="tiny_%dx%d" % (n_frames, n), xyz=xyz, sem=sem, rgb=rgb if color else None,
        edges=np.asarray(edges if edges is not None else all_pairs(n_frames),
                         dtype=np.int32).reshape(-1, 2),
        poses_gt=np.stack(gt), poses0=np.stack(init),
        params=dict(ell=ell, cutoff_mult=3.0, sigma=1.0,
                    ell_color=0.2 if color else 0.0, sem_bf16=0),
    )


def config_problem(cfg, rep=0, **kw):
    """The five benchmark workloads; seed = 1234 + 100 * cfg + rep."""
    seed = 1234 + 100 * cfg + rep
    if cfg == 1:
        return plane_sphere_problem(seed=seed, **kw)
    if cfg == 2:
        return lidar_street_problem(seed=seed, **kw)
    if cfg == 3:
        return window_problem(seed=seed, **kw)
    if cfg == 5:
        return mapping_problem(seed=seed, **kw)
    raise ValueError("config %r has no single-problem generator" % cfg)

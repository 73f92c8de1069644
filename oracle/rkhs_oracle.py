"""Plain FP64 CPU oracle of the RKHS-BA hot path.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s cpu_baseline and
``--impl reference`` legs, and by nothing else.  The CUDA library never
links, imports or calls it, and it shares no code with the CUDA path.

Everything here is slow, obvious numpy in float64, written from the paper
(Zhang et al., "RKHS-BA", arXiv 2403.01254):

  * geometric kernel  h(x, z) = sigma^2 exp(-|x - z|^2 / (2 ell^2))     Eq. (kernel), Sec. V-A
  * label inner product <l_i, l_j>, tensor product of features          Sec. III-A (label function)
  * objective F = sum_{(m,n) in C} sum_ij c_ij h(T_m x_i, T_n z_j)     Eq. (inner_product_actual_ba)
    evaluated as a sparse double sum (points far apart dropped)          Sec. III-B
  * right perturbation T exp(eps^), eps = [rho; phi], wedge            Sec. V-A (wedge operator)
  * gradient  dF/deps = -(1/ell^2) sum w (dd/deps) d,  w = c k          Eq. (inner_product_reformat), (irls_weight)
  * IRLS normal equations with frozen w, first frame fixed              Eq. (irls_gradient), (irls_final)
  * Levenberg-Marquardt on the IRLS problem, accepted while the
    original cost F increases                                           Sec. V-A (Ceres), Sec. V-C

Readings of points the paper leaves open:
  * sigma = 1 unless given; the sparse sum keeps pairs with |d|^2 < r_c^2,
    r_c = cutoff_mult * ell (strict, float64), without renormalisation.
  * c_ij = <l_i, l_j> * exp(-|c_i - c_j|^2 / (2 ell_c^2)) when colours are
    given (ell_c > 0), else <l_i, l_j>; with no labels c_ij = 1.
  * Edges are unordered pairs (a, b), a < b, each counted once.
  * loss = -F;  grad = d loss / d eps = (sigma^2 / ell^2) * b,
    b = sum w J^T d;  H = sum w J^T J (Gauss-Newton matrix of the IRLS cost),
    with d = T_a x_i - T_b y_j in world coordinates, J_a = R_a [I | -[x_i]x],
    J_b = -R_b [I | -[y_j]x]  (rho first, then phi, per the wedge).
  * RKHS distance |f_a - f_b|^2 = <f_a,f_a> + <f_b,f_b> - 2 <f_a,f_b> with the
    same sparse sums (Eq. dist_rkhs); cosine <f_a,f_b> / (|f_a| |f_b|).
  * Variants (Sec. VI time analysis, Sec. VII), off by default: pairs whose
    semantic kernel <l_i, l_j> is below sem_min are dropped; with top_k > 0
    every point of an edge's second frame keeps only its top_k pairs of
    largest w (ties: smaller index first).
  * Lengthscale decay (Sec. V-C): ell <- ell (1 - decay sign(dD/dell)) after
    each inner solve; stop when an inner solve accepts no step.
  * Rotation search (Sec. IV-A): candidate k places frame b at
    T_a [R_k | mu_a - R_k mu_b] (frame centroids aligned; the paper leaves the
    translation of a candidate open) and scores it by the cosine.
  * LM step (H_ff + lambda * Dm) delta = -b_f over every frame but frame 0,
    Dm = diag(max(H_ii, 1e-9 * max_k H_kk)); accept when F increases
    (lambda /= 10), otherwise lambda *= 10.  Stop when an accepted step has
    |delta|_inf < tol_step or relative F gain < tol_rel_f, when lambda grows
    past 1e10, or after max_iters evaluations.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import cho_factor, cho_solve
from scipy.spatial import cKDTree

__all__ = [
    "DEFAULTS", "hat", "wedge", "se3_exp", "se3_log", "pose_error",
    "label_weights", "pairs_bruteforce", "pairs_kdtree", "edge_terms",
    "evaluate", "lm_solve", "irls_frozen_solve", "edge_pairs", "select_pairs", "kernel_sums", "inner_product",
    "self_inner",
    "distance_and_cosine", "ell_decay_solve", "icosahedral_rotations", "rotation_search",
]

DEFAULTS = dict(ell=0.1, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_bf16=0,
                max_iters=100, lambda0=1e-4, tol_step=1e-10, tol_rel_f=1e-12, top_k=0, sem_min=0.0)


def _params(p):
    q = dict(DEFAULTS)
    q.update(p or {})
    return q


# ---------------------------------------------------------------------------
# SE(3): wedge, exp, log  (Sec. V-A; closed forms as in Barfoot's book)
# ---------------------------------------------------------------------------
def hat(v):
    """3x3 skew matrix [v]x with [v]x u = v x u."""
    return np.array([[0.0, -v[2], v[1]],
                     [v[2], 0.0, -v[0]],
                     [-v[1], v[0], 0.0]])


def wedge(xi):
    """4x4 matrix of the wedge operator for xi = [rho; phi] (Sec. V-A)."""
    W = np.zeros((4, 4))
    W[:3, :3] = hat(xi[3:6])
    W[:3, 3] = xi[0:3]
    return W


def se3_exp(xi):
    """exp(xi^) in closed form: R by Rodrigues, t = V rho."""
    xi = np.asarray(xi, dtype=np.float64)
    rho, phi = xi[:3], xi[3:]
    th = math.sqrt(float(phi @ phi))
    P = hat(phi)
    P2 = P @ P
    if th < 1e-5:
        # Taylor expansions of the three coefficients
        a = 1.0 - th * th / 6.0
        b = 0.5 - th * th / 24.0
        c = 1.0 / 6.0 - th * th / 120.0
    else:
        a = math.sin(th) / th
        b = (1.0 - math.cos(th)) / (th * th)
        c = (th - math.sin(th)) / (th ** 3)
    R = np.eye(3) + a * P + b * P2
    V = np.eye(3) + b * P + c * P2
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def _so3_log(R):
    """phi with exp(phi^) = R.  The angle comes from atan2 of the
    antisymmetric and trace parts (well conditioned at every angle); near pi
    the axis is read from the symmetric part S = cos(th) I + (1 - cos(th)) n n^T."""
    w = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    s = 0.5 * float(np.linalg.norm(w))            # sin(th)
    c = 0.5 * (float(np.trace(R)) - 1.0)          # cos(th)
    th = math.atan2(s, c)
    if th < 1e-5:
        return 0.5 * w * (1.0 + th * th / 6.0)
    if math.pi - th < 1e-3:
        S = 0.5 * (R + R.T)
        nn = (S - c * np.eye(3)) / (1.0 - c)
        k = int(np.argmax(np.diag(nn)))
        n = nn[:, k] / math.sqrt(nn[k, k])
        n /= np.linalg.norm(n)
        if w @ n < 0:
            n = -n
        return th * n
    return w * (th / (2.0 * s))


def se3_log(T):
    """Inverse of se3_exp: returns xi = [rho; phi]."""
    R, t = T[:3, :3], T[:3, 3]
    phi = _so3_log(R)
    th = float(np.linalg.norm(phi))
    P = hat(phi)
    if th < 1e-5:
        Vinv = np.eye(3) - 0.5 * P + (1.0 / 12.0) * (P @ P)
    else:
        half = th / 2.0
        coef = (1.0 - half * math.cos(half) / math.sin(half)) / (th * th)
        Vinv = np.eye(3) - 0.5 * P + coef * (P @ P)
    return np.concatenate([Vinv @ t, phi])


def pose_error(T_est, T_ref):
    """(rotation angle [rad], translation [m]) of T_ref^-1 T_est."""
    E = np.linalg.inv(T_ref) @ T_est
    xi = se3_log(E)
    return float(np.linalg.norm(xi[3:])), float(np.linalg.norm(E[:3, 3]))


# ---------------------------------------------------------------------------
# label inner product c_ij  (Sec. III-A)
# ---------------------------------------------------------------------------
def label_weights(sem_a, sem_b, rgb_a, rgb_b, i, j, ell_color):
    """c_ij for the pair lists i (frame a) and j (frame b)."""
    n = len(i)
    c = np.ones(n)
    if sem_a is not None:
        la = np.asarray(sem_a, dtype=np.float64)[i]
        lb = np.asarray(sem_b, dtype=np.float64)[j]
        c = np.einsum("nk,nk->n", la, lb)
    if rgb_a is not None and ell_color > 0:
        ca = np.asarray(rgb_a, dtype=np.float64)[i]
        cb = np.asarray(rgb_b, dtype=np.float64)[j]
        dc = ca - cb
        c = c * np.exp(-np.einsum("nk,nk->n", dc, dc) / (2.0 * ell_color ** 2))
    return c


# ---------------------------------------------------------------------------
# sparse double sum: pairs with |p_i - q_j|^2 < r_c^2  (Sec. III-B)
# ---------------------------------------------------------------------------
def pairs_bruteforce(p, q, rc):
    """All (i, j) with |p_i - q_j|^2 < rc^2, by the O(N^2) enumeration."""
    ii, jj = [], []
    rc2 = rc * rc
    for i0 in range(0, len(p), 256):
        d = p[i0:i0 + 256, None, :] - q[None, :, :]
        d2 = np.einsum("abk,abk->ab", d, d)
        a, b = np.nonzero(d2 < rc2)
        ii.append(a + i0)
        jj.append(b)
    if not ii:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(ii).astype(np.int64), np.concatenate(jj).astype(np.int64)


def pairs_kdtree(p, q, rc):
    """Same pair set as pairs_bruteforce: a k-d tree proposes every pair within
    a slightly larger radius, then the exact float64 test decides."""
    if len(p) == 0 or len(q) == 0 or not np.isfinite(rc):
        if np.isfinite(rc):
            return np.zeros(0, np.int64), np.zeros(0, np.int64)
        i, j = np.meshgrid(np.arange(len(p)), np.arange(len(q)), indexing="ij")
        return i.ravel().astype(np.int64), j.ravel().astype(np.int64)
    tp, tq = cKDTree(p), cKDTree(q)
    m = tp.sparse_distance_matrix(tq, rc * (1.0 + 1e-9) + 1e-12, output_type="ndarray")
    i = m["i"].astype(np.int64)
    j = m["j"].astype(np.int64)
    d = p[i] - q[j]
    keep = np.einsum("nk,nk->n", d, d) < rc * rc
    i, j = i[keep], j[keep]
    order = np.lexsort((j, i))
    return i[order], j[order]


def _hat_rows(v):
    """[v_n]x for every row v_n of v, shape (n, 3, 3)."""
    n = len(v)
    z = np.zeros(n)
    return np.stack([np.stack([z, -v[:, 2], v[:, 1]], 1),
                     np.stack([v[:, 2], z, -v[:, 0]], 1),
                     np.stack([-v[:, 1], v[:, 0], z], 1)], 1)


def _transform(T, x):
    return x @ T[:3, :3].T + T[:3, 3]


# ---------------------------------------------------------------------------
# per-edge terms: F, b = sum w J^T d, H = sum w J^T J   (Sec. V-A)
# ---------------------------------------------------------------------------
def edge_terms(xa, xb, Ta, Tb, sem_a=None, sem_b=None, rgb_a=None, rgb_b=None,
               params=None, enumerate_pairs=pairs_kdtree, chunk=200000):
    """Contribution of one edge (a, b).

    Returns dict(F, E, n_pairs, b (12,), H (12, 12)) with b, H ordered
    [rho_a, phi_a, rho_b, phi_b].  F = sigma^2 sum w, E = sum w |d|^2.
    """
    P = _params(params)
    ell, sigma = P["ell"], P["sigma"]
    rc = P["cutoff_mult"] * ell
    xa = np.asarray(xa, np.float64)
    xb = np.asarray(xb, np.float64)
    p = _transform(Ta, xa)          # T_a x_i
    q = _transform(Tb, xb)          # T_b y_j
    i, j = enumerate_pairs(p, q, rc)
    if P["sem_min"] > 0 or P["top_k"] > 0:
        keep = select_pairs(p, q, i, j, sem_a, sem_b, rgb_a, rgb_b, P)
        i, j = i[keep], j[keep]
    out = dict(F=0.0, E=0.0, n_pairs=int(len(i)), b=np.zeros(12), H=np.zeros((12, 12)),
               W=0.0)
    Ra, Rb = Ta[:3, :3], Tb[:3, :3]
    for s in range(0, len(i), chunk):
        ii, jj = i[s:s + chunk], j[s:s + chunk]
        d = p[ii] - q[jj]                                   # world-frame residual
        d2 = np.einsum("nk,nk->n", d, d)
        c = label_weights(sem_a, sem_b, rgb_a, rgb_b, ii, jj, P["ell_color"])
        w = c * np.exp(-d2 / (2.0 * ell * ell))             # Eq. (irls_weight)
        n = len(ii)
        # J_a = R_a [I | -[x]x],  J_b = -R_b [I | -[y]x]
        Ax = np.zeros((n, 3, 6))
        Ay = np.zeros((n, 3, 6))
        Ax[:, :, :3] = np.eye(3)
        Ay[:, :, :3] = np.eye(3)
        Ax[:, :, 3:] = -_hat_rows(xa[ii])
        Ay[:, :, 3:] = -_hat_rows(xb[jj])
        J = np.concatenate([np.einsum("ij,njk->nik", Ra, Ax),
                            -np.einsum("ij,njk->nik", Rb, Ay)], axis=2)   # (n, 3, 12)
        out["F"] += sigma * sigma * float(w.sum())
        out["W"] += float(w.sum())
        out["E"] += float((w * d2).sum())
        out["b"] += np.einsum("nki,nk->i", J, w[:, None] * d)
        Jf = J.reshape(-1, 12)
        out["H"] += (Jf * np.repeat(w, 3)[:, None]).T @ Jf
    return out


def select_pairs(p, q, i, j, sem_a, sem_b, rgb_a, rgb_b, P):
    """Variants of the sparse sum (Sec. VI time analysis, Sec. VII): drop the
    pairs whose semantic kernel <l_i, l_j> is below sem_min, then keep for
    every point j of the edge's second frame only the top_k pairs with the
    largest weight w (ties: smaller i first).  Returns a boolean mask."""
    keep = np.ones(len(i), dtype=bool)
    if P["sem_min"] > 0 and sem_a is not None:
        la = np.asarray(sem_a, dtype=np.float64)[i]
        lb = np.asarray(sem_b, dtype=np.float64)[j]
        keep &= np.einsum("nk,nk->n", la, lb) >= P["sem_min"]
    if P["top_k"] > 0 and len(i):
        d = p[i] - q[j]
        w = label_weights(sem_a, sem_b, rgb_a, rgb_b, i, j, P["ell_color"]) * \
            np.exp(-np.einsum("nk,nk->n", d, d) / (2.0 * P["ell"] ** 2))
        idx = np.nonzero(keep)[0]
        order = idx[np.lexsort((i[idx], -w[idx], j[idx]))]       # by j, then w descending, then i
        jj = j[order]
        first = np.r_[True, jj[1:] != jj[:-1]]
        start = np.maximum.accumulate(np.where(first, np.arange(len(jj)), 0))
        rank = np.arange(len(jj)) - start
        keep[:] = False
        keep[order[rank < P["top_k"]]] = True
    return keep


def edge_pairs(problem, poses, e, enumerate_pairs=pairs_kdtree):
    """(i, j) index arrays of the pairs of edge e at the given poses."""
    a, b = (int(v) for v in problem["edges"][e])
    P = _params(problem["params"])
    p = _transform(poses[a], np.asarray(problem["xyz"][a], np.float64))
    q = _transform(poses[b], np.asarray(problem["xyz"][b], np.float64))
    return enumerate_pairs(p, q, P["cutoff_mult"] * P["ell"])


def _frame_inputs(problem, m):
    sem = problem.get("sem")
    rgb = problem.get("rgb")
    return (problem["xyz"][m], None if sem is None else sem[m],
            None if rgb is None else rgb[m])


def evaluate(problem, poses, edge_subset=None, enumerate_pairs=pairs_kdtree, params=None):
    """loss = -F, grad = d loss/d eps (6K), H_full = sum w J^T J (6K x 6K),
    per-edge 12x12 blocks, pair counts; all float64."""
    P = _params(problem["params"])
    if params:
        P.update(params)
    K = len(problem["xyz"])
    edges = np.asarray(problem["edges"]).reshape(-1, 2)
    sel = range(len(edges)) if edge_subset is None else edge_subset
    F = 0.0
    E = 0.0
    b = np.zeros(6 * K)
    H = np.zeros((6 * K, 6 * K))
    blocks, per_edge_pairs, per_edge_F, per_edge_b = [], [], [], []
    for e in sel:
        a, bb = (int(v) for v in edges[e])
        xa, sa, ca = _frame_inputs(problem, a)
        xb, sb, cb = _frame_inputs(problem, bb)
        t = edge_terms(xa, xb, poses[a], poses[bb], sa, sb, ca, cb, P,
                       enumerate_pairs=enumerate_pairs)
        F += t["F"]
        E += t["E"]
        idx = np.r_[6 * a:6 * a + 6, 6 * bb:6 * bb + 6]
        b[idx] += t["b"]
        H[np.ix_(idx, idx)] += t["H"]
        blocks.append(t["H"])
        per_edge_pairs.append(t["n_pairs"])
        per_edge_F.append(t["F"])
        per_edge_b.append(t["b"])
    scale = P["sigma"] ** 2 / P["ell"] ** 2
    return dict(loss=-F, F=F, E=E, grad=scale * b, b=b, H=H,
                H_blocks=np.array(blocks).reshape(-1, 12, 12),
                edge_pairs=np.array(per_edge_pairs, dtype=np.int64),
                edge_F=np.array(per_edge_F), edge_b=np.array(per_edge_b).reshape(-1, 12),
                n_pairs=int(sum(per_edge_pairs)))


# ---------------------------------------------------------------------------
# Levenberg-Marquardt on the IRLS problem (Sec. V-A, V-C)
# ---------------------------------------------------------------------------
def _lm_delta(H, b, lam):
    """Solve (H_ff + lam * Dm) delta = -b_f; frame 0 (first 6 DOF) is fixed."""
    Hf = H[6:, 6:]
    bf = b[6:]
    dg = np.diag(Hf).copy()
    floor = 1e-9 * max(float(dg.max()) if dg.size else 0.0, 1e-300)
    A = Hf + lam * np.diag(np.maximum(dg, floor))
    delta = -cho_solve(cho_factor(A), bf)
    return np.concatenate([np.zeros(6), delta])


def _retract(poses, delta):
    out = poses.copy()
    for m in range(1, len(poses)):
        out[m] = poses[m] @ se3_exp(delta[6 * m:6 * m + 6])
    return out


def lm_solve(problem, poses0=None, params=None, enumerate_pairs=pairs_kdtree,
             evaluate_fn=None):
    """Damped Gauss-Newton on the IRLS cost; weights recomputed each step.

    Returns dict(poses, F, iters (evaluations after the first), status,
    n_pairs_total, history)."""
    P = _params(problem["params"])
    if params:
        P.update(params)
    ev = evaluate_fn or (lambda T: evaluate(problem, T, enumerate_pairs=enumerate_pairs,
                                            params=P))
    T = np.array(problem["poses0"] if poses0 is None else poses0, dtype=np.float64)
    cur = ev(T)
    lam = P["lambda0"]
    n_pairs = cur["n_pairs"]
    status = "max_iters"
    history = [cur["F"]]
    it = 0
    while it < P["max_iters"]:
        delta = _lm_delta(cur["H"], cur["b"], lam)
        Tc = _retract(T, delta)
        cand = ev(Tc)
        it += 1
        n_pairs += cand["n_pairs"]
        step = float(np.abs(delta).max())
        if cand["F"] > cur["F"]:
            rel = (cand["F"] - cur["F"]) / max(abs(cur["F"]), 1e-300)
            T, cur = Tc, cand
            lam = max(lam / 10.0, 1e-12)
            history.append(cur["F"])
            if step < P["tol_step"] or rel < P["tol_rel_f"]:
                status = "converged"
                break
        else:
            lam *= 10.0
            if step < P["tol_step"] or lam > 1e10:
                status = "converged"
                break
    return dict(poses=T, F=cur["F"], iters=it, status=status, n_pairs_total=n_pairs,
                history=history, lam=lam)


def irls_frozen_solve(xa, xb, i, j, w, Ta, Tb, iters=50, lam=0.0):
    """Minimise sum w |T_a x_i - T_b y_j|^2 over T_b with T_a and w fixed
    (Eq. (irls_final) for one edge), by the same Gauss-Newton blocks."""
    Tb = Tb.copy()
    xa = np.asarray(xa, np.float64)
    xb = np.asarray(xb, np.float64)
    Ra = Ta[:3, :3]
    for _ in range(iters):
        p = _transform(Ta, xa[i])
        q = _transform(Tb, xb[j])
        d = p - q
        Rb = Tb[:3, :3]
        y = xb[j]
        n = len(i)
        Ay = np.zeros((n, 3, 6))
        Ay[:, :, :3] = np.eye(3)
        Ay[:, :, 3:] = -_hat_rows(y)
        Jb = -np.einsum("ij,njk->nik", Rb, Ay)
        bb = np.einsum("nki,nk->i", Jb, w[:, None] * d)
        Jf = Jb.reshape(-1, 6)
        Hb = (Jf * np.repeat(w, 3)[:, None]).T @ Jf
        delta = -np.linalg.solve(Hb + lam * np.diag(np.diag(Hb)), bb)
        Tb = Tb @ se3_exp(delta)
        if np.abs(delta).max() < 1e-14:
            break
    del Ra
    return Tb


# ---------------------------------------------------------------------------
# inner products, RKHS distance and cosine (Sec. III-A, Eq. dist_rkhs)
# ---------------------------------------------------------------------------
def kernel_sums(xa, xb, Ta, Tb, sem_a=None, sem_b=None, rgb_a=None, rgb_b=None, params=None, chunk=500000):
    """F = sigma^2 sum w and E = sum w |d|^2 over the pairs inside the cutoff,
    w = c k (no Jacobians: the function-space quantities need only these)."""
    P = _params(params)
    ell, sigma = P["ell"], P["sigma"]
    p = _transform(Ta, np.asarray(xa, np.float64))
    q = _transform(Tb, np.asarray(xb, np.float64))
    i, j = pairs_kdtree(p, q, P["cutoff_mult"] * ell)
    if P["sem_min"] > 0 or P["top_k"] > 0:
        keep = select_pairs(p, q, i, j, sem_a, sem_b, rgb_a, rgb_b, P)
        i, j = i[keep], j[keep]
    F = E = 0.0
    for s in range(0, len(i), chunk):
        ii, jj = i[s:s + chunk], j[s:s + chunk]
        d = p[ii] - q[jj]
        d2 = np.einsum("nk,nk->n", d, d)
        w = label_weights(sem_a, sem_b, rgb_a, rgb_b, ii, jj, P["ell_color"]) * np.exp(-d2 / (2.0 * ell * ell))
        F += sigma * sigma * float(w.sum())
        E += float((w * d2).sum())
    return dict(F=F, E=E, n_pairs=int(len(i)))


def inner_product(xa, xb, Ta, Tb, sem_a=None, sem_b=None, rgb_a=None, rgb_b=None, params=None):
    """<f_{T_a X_a}, f_{T_b X_b}> over the pairs inside the cutoff (Eq. double_sum)."""
    return kernel_sums(xa, xb, Ta, Tb, sem_a, sem_b, rgb_a, rgb_b, params)["F"]


def self_inner(x, sem=None, rgb=None, params=None):
    """<f_X, f_X>: the double sum of a frame with itself (pose invariant)."""
    I = np.eye(4)
    return inner_product(x, x, I, I, sem, sem, rgb, rgb, params)


def distance_and_cosine(problem, poses, params=None):
    """Per edge: RKHS distance |f_a - f_b|^2 = <f_a,f_a> + <f_b,f_b> - 2<f_a,f_b>
    (Eq. dist_rkhs) and the cosine <f_a,f_b> / (|f_a| |f_b|); the self terms;
    and d(sum of the edge distances)/d ell.  Each inner product is
    sigma^2 sum c k with k = exp(-|d|^2 / 2 ell^2), so its derivative in ell
    is sigma^2 / ell^3 sum c k |d|^2 (the moving cutoff is not differentiated)."""
    P = _params(problem["params"])
    if params:
        P.update(params)
    K = len(problem["xyz"])
    I = np.eye(4)
    s_terms = []
    for m in range(K):
        x, s, c = _frame_inputs(problem, m)
        s_terms.append(kernel_sums(x, x, I, I, s, s, c, c, P))
    selfs = np.array([t["F"] for t in s_terms])
    self_E = np.array([t["E"] for t in s_terms])
    dist, cos, cross, cross_E = [], [], [], []
    for a, b in np.asarray(problem["edges"]).reshape(-1, 2):
        a, b = int(a), int(b)
        xa, sa, ca = _frame_inputs(problem, a)
        xb, sb, cb = _frame_inputs(problem, b)
        t = kernel_sums(xa, xb, poses[a], poses[b], sa, sb, ca, cb, P)
        cross.append(t["F"])
        cross_E.append(t["E"])
        dist.append(selfs[a] + selfs[b] - 2.0 * t["F"])
        cos.append(t["F"] / math.sqrt(selfs[a] * selfs[b]) if selfs[a] > 0 and selfs[b] > 0 else 0.0)
    sig2, ell = P["sigma"] ** 2, P["ell"]
    dE = sum(self_E[int(a)] + self_E[int(b)] for a, b in np.asarray(problem["edges"]).reshape(-1, 2))
    dD_dell = sig2 / ell ** 3 * (dE - 2.0 * float(np.sum(cross_E)))
    return dict(self=selfs, cross=np.array(cross), dist=np.array(dist), cos=np.array(cos),
                self_E=self_E, cross_E=np.array(cross_E), dD_dell=dD_dell)


def ell_decay_solve(problem, poses0=None, params=None, decay=0.1, ell_min=0.0, max_outer=10):
    """Inner-outer loop of Sec. V-C.  Inner: the LM pose solve at fixed ell.
    Outer: ell <- ell (1 - decay * sign(dD/dell)), D the summed edge distance
    of Eq. dist_rkhs at the solved poses, floored at ell_min.  The loop ends
    when an inner solve accepts no step (the original objective stops
    increasing), when ell stops changing, or after max_outer levels."""
    P = _params(problem["params"])
    if params:
        P.update(params)
    T = np.array(problem["poses0"] if poses0 is None else poses0, dtype=np.float64)
    ell = P["ell"]
    levels = []
    for _ in range(max_outer):
        Q = dict(P, ell=ell)
        r = lm_solve(problem, T, params=Q)
        T = r["poses"]
        g = distance_and_cosine(problem, T, params=Q)["dD_dell"]
        accepted = len(r["history"]) - 1
        levels.append(dict(ell=ell, F=r["F"], iters=r["iters"], accepted=accepted, dD_dell=g))
        if accepted == 0:
            break
        nxt = max(ell * (1.0 - decay * float(np.sign(g))), ell_min)
        if nxt == ell:
            break
        ell = nxt
    return dict(poses=T, ell=ell, levels=levels)


# ---------------------------------------------------------------------------
# icosahedral rotation search (Sec. IV-A)
# ---------------------------------------------------------------------------
def _axis_rotation(axis, angle):
    axis = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    return se3_exp(np.concatenate([np.zeros(3), angle * axis]))[:3, :3]


def icosahedral_rotations():
    """The 60 rotations of the icosahedron's symmetry group, built as the
    paper lists them: the identity; a half turn about each of the 15 axes
    through midpoints of opposite edges; turns of 2pi/3 and 4pi/3 about each
    of the 10 axes through centres of opposite faces; turns of 2k pi/5,
    k = 1..4, about each of the 6 axes through opposite vertices."""
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    V = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            V += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    V = np.array(V)
    edge_len = min(np.linalg.norm(V[i] - V[j]) for i in range(12) for j in range(i + 1, 12))
    edges = [(i, j) for i in range(12) for j in range(i + 1, 12)
             if abs(np.linalg.norm(V[i] - V[j]) - edge_len) < 1e-9]
    faces = [(i, j, k) for (i, j) in edges for k in range(j + 1, 12)
             if (i, k) in edges and (j, k) in edges]

    def half(dirs):
        out = []
        for d in dirs:
            d = d / np.linalg.norm(d)
            if not any(abs(abs(d @ e) - 1.0) < 1e-9 for e in out):
                out.append(d)
        return out

    v_axes = half(list(V))
    e_axes = half([V[i] + V[j] for i, j in edges])
    f_axes = half([V[i] + V[j] + V[k] for i, j, k in faces])
    R = [np.eye(3)]
    R += [_axis_rotation(a, math.pi) for a in e_axes]
    R += [_axis_rotation(a, t * 2 * math.pi / 3) for a in f_axes for t in (1, 2)]
    R += [_axis_rotation(a, t * 2 * math.pi / 5) for a in v_axes for t in (1, 2, 3, 4)]
    return np.array(R)


def rotation_search(problem, a, b, poses, params=None):
    """Score the 60 candidate rotations of frame b against frame a: candidate k
    places b at T_a [R_k | mu_a - R_k mu_b] (centroids aligned); the score is
    the cosine of Sec. IV-A.  Returns (cosines [60], best pose of b)."""
    P = _params(problem["params"])
    if params:
        P.update(params)
    xa, sa, ca = _frame_inputs(problem, a)
    xb, sb, cb = _frame_inputs(problem, b)
    xa = np.asarray(xa, np.float64)
    xb = np.asarray(xb, np.float64)
    Sa = self_inner(xa, sa, ca, P)
    Sb = self_inner(xb, sb, cb, P)
    mua, mub = xa.mean(0), xb.mean(0)
    cos = np.zeros(60)
    cands = []
    for k, Rk in enumerate(icosahedral_rotations()):
        C = np.eye(4)
        C[:3, :3] = Rk
        C[:3, 3] = mua - Rk @ mub
        Tb = poses[a] @ C
        cands.append(Tb)
        cos[k] = inner_product(xa, xb, poses[a], Tb, sa, sb, ca, cb, P) / math.sqrt(Sa * Sb)
    return cos, cands[int(np.argmax(cos))]

"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: derivatives are checked by
finite differences of the objective or of the residual, SE(3) exp against the
matrix exponential of the wedge matrix, the frozen-weight IRLS minimiser
against the weighted Procrustes (Kabsch/Horn) closed form, pair sets against
O(N^2) enumeration, label weighting against pure-Python loops, and gauge
freedom against the 6-dimensional null space it must produce.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm, logm

import oracle as O
import scenes

RNG = np.random.default_rng(20240301)


def _rand_xi(rng, rot=1.0, trans=1.0):
    return np.concatenate([rng.normal(size=3) * trans, rng.normal(size=3) * rot])


# ---------------------------------------------------------------- SE(3) -----
@pytest.mark.parametrize("scale", [1e-9, 1e-6, 1e-3, 0.1, 1.0, 2.5])
def test_se3_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(1)
    for _ in range(5):
        xi = _rand_xi(rng) * scale
        np.testing.assert_allclose(O.se3_exp(xi), expm(O.wedge(xi)), atol=1e-13, rtol=0)


def test_wedge_layout_is_the_papers():
    # Sec. V-A: rows [0 -phi3 phi2 rho1; phi3 0 -phi1 rho2; -phi2 phi1 0 rho3; 0 0 0 0]
    W = O.wedge(np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0]))
    np.testing.assert_array_equal(W, [[0, -6, 5, 1], [6, 0, -4, 2], [-5, 4, 0, 3], [0, 0, 0, 0]])


@pytest.mark.parametrize("angle", [0.0, 1e-8, 1e-4, 0.3, 2.0, math.pi - 1e-3, math.pi - 1e-6])
def test_se3_log_inverts_exp(angle):
    rng = np.random.default_rng(2)
    for _ in range(4):
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        xi = np.concatenate([rng.normal(size=3), angle * ax])
        back = O.se3_log(O.se3_exp(xi))
        np.testing.assert_allclose(O.se3_exp(back), O.se3_exp(xi), atol=1e-9)
        if angle < math.pi - 1e-2:
            np.testing.assert_allclose(back, xi, atol=1e-9)


def test_se3_log_matches_matrix_logarithm():
    rng = np.random.default_rng(3)
    for _ in range(5):
        T = scenes.random_pose(rng, rng.uniform(1, 150), rng.uniform(0, 3))
        L = np.real(logm(T))
        xi = O.se3_log(T)
        np.testing.assert_allclose(O.wedge(xi), L, atol=1e-10)


# ---------------------------------------------------------- pair sets -------
def test_kdtree_pairs_equal_bruteforce():
    rng = np.random.default_rng(4)
    for n, m, rc in ((50, 70, 0.2), (300, 200, 0.15), (1, 400, 0.5), (0, 10, 0.3)):
        p = rng.uniform(0, 1, size=(n, 3))
        q = rng.uniform(0, 1, size=(m, 3))
        a = O.pairs_bruteforce(p, q, rc)
        b = O.pairs_kdtree(p, q, rc)
        sa = set(zip(a[0].tolist(), a[1].tolist()))
        sb = set(zip(b[0].tolist(), b[1].tolist()))
        assert sa == sb


def test_cutoff_is_strict_and_at_r_c():
    ell = 0.1
    rc = 3 * ell
    for frac, present in ((0.999, True), (1.001, False)):
        prob = dict(xyz=[np.zeros((1, 3)), np.array([[frac * rc, 0.0, 0.0]])], sem=None,
                    rgb=None, edges=np.array([[0, 1]]), params=dict(ell=ell))
        r = O.evaluate(prob, np.stack([np.eye(4)] * 2))
        assert (r["n_pairs"] == 1) == present


def test_single_pair_value():
    # two frames holding one point each; F = s * exp(-|d|^2 / 2 ell^2)
    ell = 0.2
    prob = dict(xyz=[np.array([[0.1, -0.2, 0.3]]), np.array([[0.0, 0.0, 0.0]])],
                sem=[np.array([[0.25, 0.75]]), np.array([[0.5, 0.5]])], rgb=None,
                edges=np.array([[0, 1]]), params=dict(ell=ell, sigma=1.5))
    T1 = scenes.make_pose(np.eye(3), np.array([0.05, -0.1, 0.2]))
    r = O.evaluate(prob, np.stack([np.eye(4), T1]))
    d2 = 0.05 ** 2 + 0.1 ** 2 + 0.1 ** 2
    assert r["n_pairs"] == 1
    assert abs(r["F"] - 1.5 ** 2 * 0.5 * math.exp(-d2 / (2 * ell * ell))) < 1e-15


# ------------------------------------------ label weighting, brute force ----
def _loop_F(prob, poses):
    """Pure-Python double loop over every edge and point pair (tiny inputs)."""
    P = dict(O.DEFAULTS)
    P.update(prob["params"])
    rc2 = (P["cutoff_mult"] * P["ell"]) ** 2
    F = 0.0
    for a, b in prob["edges"]:
        Ta, Tb = poses[a], poses[b]
        for i, x in enumerate(prob["xyz"][a]):
            px = Ta[:3, :3] @ x + Ta[:3, 3]
            for j, y in enumerate(prob["xyz"][b]):
                qy = Tb[:3, :3] @ y + Tb[:3, 3]
                d2 = float(sum((px[k] - qy[k]) ** 2 for k in range(3)))
                if d2 >= rc2:
                    continue
                c = 1.0
                if prob.get("sem") is not None:
                    c = sum(float(u) * float(v) for u, v in zip(prob["sem"][a][i], prob["sem"][b][j]))
                if prob.get("rgb") is not None and P["ell_color"] > 0:
                    dc = sum((float(u) - float(v)) ** 2 for u, v in zip(prob["rgb"][a][i], prob["rgb"][b][j]))
                    c *= math.exp(-dc / (2 * P["ell_color"] ** 2))
                F += P["sigma"] ** 2 * c * math.exp(-d2 / (2 * P["ell"] ** 2))
    return F


@pytest.mark.parametrize("color", [False, True])
def test_objective_equals_python_double_loop(color):
    prob = scenes.tiny_problem(seed=11, n_frames=3, n=25, color=color)
    F_loop = _loop_F(prob, prob["poses0"])
    r = O.evaluate(prob, prob["poses0"])
    assert r["n_pairs"] > 20
    assert abs(r["F"] - F_loop) <= 1e-12 * abs(F_loop)


def test_one_hot_labels_keep_only_same_class_pairs():
    rng = np.random.default_rng(5)
    n = 40
    base = rng.uniform(0, 0.6, size=(n, 3))
    la, lb = rng.integers(0, 3, n), rng.integers(0, 3, n)
    prob = dict(xyz=[base, base + 0.01], sem=[scenes.one_hot(la, 3), scenes.one_hot(lb, 3)],
                rgb=None, edges=np.array([[0, 1]]), params=dict(ell=0.1))
    poses = np.stack([np.eye(4)] * 2)
    r = O.evaluate(prob, poses)
    plain = dict(prob, sem=None)
    i, j = O.edge_pairs(plain, poses, 0)
    d = base[i] - (base[j] + 0.01)
    k = np.exp(-np.einsum("nk,nk->n", d, d) / (2 * 0.01))
    assert abs(r["F"] - k[la[i] == lb[j]].sum()) < 1e-12
    # without labels the sum is plain kernel correlation (Sec. III-A)
    assert abs(O.evaluate(plain, poses)["F"] - k.sum()) < 1e-12


# ------------------------------------------------------- derivatives --------
def _all_pairs_problem(seed=6, n_frames=3, n=20, color=True):
    prob = scenes.tiny_problem(seed=seed, n_frames=n_frames, n=n, color=color)
    prob["params"] = dict(prob["params"], cutoff_mult=np.inf, sigma=1.3)
    return prob


def _perturbed(poses, m, k, h):
    out = poses.copy()
    e = np.zeros(6)
    e[k] = h
    out[m] = poses[m] @ O.se3_exp(e)
    return out


def test_gradient_matches_finite_differences():
    prob = _all_pairs_problem()
    T = prob["poses0"]
    r = O.evaluate(prob, T)
    h = 1e-6
    fd = np.zeros_like(r["grad"])
    for m in range(len(T)):
        for k in range(6):
            lp = O.evaluate(prob, _perturbed(T, m, k, h))["loss"]
            lm = O.evaluate(prob, _perturbed(T, m, k, -h))["loss"]
            fd[6 * m + k] = (lp - lm) / (2 * h)
    assert np.linalg.norm(r["grad"] - fd) <= 1e-6 * np.linalg.norm(fd)


def test_gauss_newton_blocks_match_finite_difference_jacobians():
    prob = _all_pairs_problem(n=12, n_frames=2)
    T = prob["poses0"]
    r = O.evaluate(prob, T)
    xa, xb = prob["xyz"][0], prob["xyz"][1]
    P = dict(O.DEFAULTS)
    P.update(prob["params"])
    h = 1e-6
    H = np.zeros((12, 12))
    b = np.zeros(12)

    def resid(Ta, Tb, i, j):
        return (Ta[:3, :3] @ xa[i] + Ta[:3, 3]) - (Tb[:3, :3] @ xb[j] + Tb[:3, 3])

    for i in range(len(xa)):
        for j in range(len(xb)):
            d = resid(T[0], T[1], i, j)
            c = float(prob["sem"][0][i] @ prob["sem"][1][j].astype(np.float64))
            dc = prob["rgb"][0][i].astype(np.float64) - prob["rgb"][1][j]
            c *= math.exp(-float(dc @ dc) / (2 * P["ell_color"] ** 2))
            w = c * math.exp(-float(d @ d) / (2 * P["ell"] ** 2))
            J = np.zeros((3, 12))
            for col in range(12):
                m, k = divmod(col, 6)
                Tp = _perturbed(T, m, k, h)
                Tm = _perturbed(T, m, k, -h)
                J[:, col] = (resid(Tp[0], Tp[1], i, j) - resid(Tm[0], Tm[1], i, j)) / (2 * h)
            H += w * J.T @ J
            b += w * J.T @ d
    np.testing.assert_allclose(r["H"], H, atol=1e-7 * np.abs(H).max())
    np.testing.assert_allclose(r["b"], b, atol=1e-7 * np.abs(b).max())
    # grad = (sigma^2 / ell^2) b : the factor of Eq. (inner_product_reformat)
    np.testing.assert_allclose(r["grad"], P["sigma"] ** 2 / P["ell"] ** 2 * r["b"], rtol=1e-14)


def test_hessian_is_psd_and_weights_bounded():
    prob = scenes.tiny_problem(seed=8, n_frames=3, n=50)
    r = O.evaluate(prob, prob["poses0"])
    ev = np.linalg.eigvalsh(r["H"])
    assert ev.min() >= -1e-10 * ev.max()
    # 0 <= w <= 1 for probability labels (Sec. V-B): F <= sigma^2 * n_pairs
    assert 0 <= r["F"] <= r["n_pairs"]


# ---------------------------------------------------- invariances -----------
def _adjoint(T):
    R, t = T[:3, :3], T[:3, 3]
    A = np.zeros((6, 6))
    A[:3, :3] = R
    A[:3, 3:] = O.hat(t) @ R
    A[3:, 3:] = R
    return A


def test_gauge_invariance_and_null_space():
    prob = scenes.tiny_problem(seed=9, n_frames=4, n=40)
    prob["params"] = dict(prob["params"], cutoff_mult=np.inf)
    T = prob["poses0"]
    r = O.evaluate(prob, T)
    G = scenes.random_pose(np.random.default_rng(10), 37.0, 2.0)
    r2 = O.evaluate(prob, np.stack([G @ Tm for Tm in T]))
    assert abs(r2["F"] - r["F"]) <= 1e-12 * abs(r["F"])
    rng = np.random.default_rng(11)
    for rot in (0.0, 1.0):
        for _ in range(4):
            xi = np.concatenate([rng.normal(size=3), rot * rng.normal(size=3)])
            v = np.concatenate([_adjoint(np.linalg.inv(Tm)) @ xi for Tm in T])
            # F is invariant under a common left motion, so the gradient is
            # orthogonal to all six gauge directions ...
            assert abs(r["grad"] @ v) <= 1e-9 * np.linalg.norm(r["grad"]) * np.linalg.norm(v)
            Hv = np.linalg.norm(r["H"] @ v)
            if rot == 0.0:
                # ... and a common translation leaves every residual unchanged,
                # so it lies in the null space of sum w J^T J; a common rotation
                # rotates the residuals (J v = phi x d) and does not.
                assert Hv <= 1e-9 * np.linalg.norm(r["H"]) * np.linalg.norm(v)
            else:
                assert Hv > 1e-6 * np.linalg.norm(r["H"]) * np.linalg.norm(v)


def test_edge_direction_does_not_matter():
    prob = scenes.tiny_problem(seed=12, n_frames=2, n=60)
    T = prob["poses0"]
    F = O.evaluate(prob, T)["F"]
    swapped = dict(prob, xyz=prob["xyz"][::-1], sem=prob["sem"][::-1])
    assert abs(O.evaluate(swapped, T[::-1])["F"] - F) <= 1e-12 * F


def test_identical_clouds_at_identity_have_zero_gradient():
    prob = scenes.tiny_problem(seed=13, n_frames=2, n=80)
    prob["xyz"][1] = prob["xyz"][0].copy()
    prob["sem"][1] = prob["sem"][0].copy()
    r = O.evaluate(prob, np.stack([np.eye(4)] * 2))
    assert r["n_pairs"] > 80
    assert np.abs(r["grad"]).max() <= 1e-10 * np.abs(r["H"]).max()


# ------------------------------------------------------- solver -------------
def _kabsch(x, y, w):
    """Weighted Procrustes: R, t minimising sum w |x - (R y + t)|^2."""
    ws = w / w.sum()
    mx, my = ws @ x, ws @ y
    C = ((x - mx) * ws[:, None]).T @ (y - my)
    U, _, Vt = np.linalg.svd(C)
    D = np.diag([1.0, 1.0, np.linalg.det(U @ Vt)])
    R = U @ D @ Vt
    return R, mx - R @ my


def test_frozen_weight_irls_reaches_weighted_kabsch():
    rng = np.random.default_rng(14)
    x = rng.uniform(-1, 1, size=(200, 3))
    Tgt = scenes.random_pose(rng, 25.0, 0.4)
    y = scenes.to_local(x, Tgt) + rng.normal(scale=0.03, size=x.shape)
    i = np.arange(200)
    w = rng.uniform(0.05, 1.0, size=200)
    Tb = O.irls_frozen_solve(x, y, i, i, w, np.eye(4), np.eye(4), iters=100)
    R, t = _kabsch(x, y, w)
    np.testing.assert_allclose(Tb[:3, :3], R, atol=1e-10)
    np.testing.assert_allclose(Tb[:3, 3], t, atol=1e-10)


def test_lm_recovers_ground_truth_on_identical_clouds():
    prob = scenes.plane_sphere_problem(seed=15, n=1500, same_points=True, angle_deg=2.0,
                                       trans=0.04, ell=0.1)
    res = O.lm_solve(prob, params=dict(max_iters=60))
    dr, dt = O.pose_error(res["poses"][1], prob["poses_gt"][1])
    assert res["status"] == "converged"
    assert dr < 1e-6 and dt < 1e-6
    # the objective only increases along accepted steps (Sec. V-C)
    assert all(b >= a for a, b in zip(res["history"], res["history"][1:]))


def test_lm_stationary_point_has_vanishing_irls_gradient():
    # all-pairs (no cutoff): the truncated sum jumps when pairs cross r_c, so
    # only the smooth objective has a stationary point in the strict sense
    prob = scenes.tiny_problem(seed=16, n_frames=3, n=120, max_deg=3.0, max_trans=0.03)
    prob["params"] = dict(prob["params"], cutoff_mult=np.inf)
    res = O.lm_solve(prob, params=dict(max_iters=80))
    assert res["status"] == "converged"
    r = O.evaluate(prob, res["poses"])
    # Eq. (irls_gradient): sum w (dd/deps) d = 0 for every free frame
    assert np.abs(r["b"][6:]).max() <= 1e-7 * np.abs(r["H"]).max()


# --------------------------------------------------- degenerate cases -------
def test_empty_frame_and_no_pairs():
    prob = dict(xyz=[np.zeros((0, 3)), np.ones((5, 3))], sem=None, rgb=None,
                edges=np.array([[0, 1]]), params=dict(ell=0.1))
    r = O.evaluate(prob, np.stack([np.eye(4)] * 2))
    assert r["n_pairs"] == 0 and r["F"] == 0 and not r["H"].any()
    far = dict(prob, xyz=[np.zeros((3, 3)), np.full((5, 3), 10.0)])
    assert O.evaluate(far, np.stack([np.eye(4)] * 2))["n_pairs"] == 0


def test_bf16_rounding_of_inputs_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(17).dirichlet(np.full(19, 0.3), size=500).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).float().numpy()
    np.testing.assert_array_equal(scenes.round_to_bf16(a), ref)

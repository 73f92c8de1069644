"""Pins of the oracle's RKHS distance, cosine, lengthscale derivative and
icosahedral rotation search (Sec. III-A Eq. dist_rkhs, Sec. IV-A, Sec. V-C).

Each pin checks the oracle against something other than itself: the closed
form of one pair, the L2 norm of the Gaussian-smoothed point functions by
quadrature (the RKHS distance of a Gaussian kernel), positive definiteness,
central differences in ell, group axioms of the rotation set and the exact
recovery of a rotation that lies in the group.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

ALL = dict(cutoff_mult=math.inf)          # every pair counts: no truncation


def _problem(xyz, edges, ell=0.2, sem=None, **kw):
    p = dict(xyz=[np.asarray(x, np.float64) for x in xyz], edges=np.asarray(edges, np.int32).reshape(-1, 2),
             params=dict(ell=ell, sigma=1.0, **kw), poses0=np.stack([np.eye(4)] * len(xyz)))
    if sem is not None:
        p["sem"] = [np.asarray(s, np.float32) for s in sem]
        p["params"]["sem_dim"] = p["sem"][0].shape[1]
    return p


# ------------------------------------------------------- rotation group -----
def _icosahedron_vertices():
    phi = (1 + 5 ** 0.5) / 2
    V = []
    for s1, s2 in itertools.product((-1, 1), repeat=2):
        V += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    return np.array(V, np.float64)


def test_icosahedral_set_is_the_rotation_group_of_the_icosahedron():
    R = O.icosahedral_rotations()
    assert R.shape == (60, 3, 3)
    for r in R:
        np.testing.assert_allclose(r @ r.T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(r) - 1) < 1e-13
    flat = R.reshape(60, 9)
    dmin = min(np.abs(flat[i] - flat[j]).max() for i in range(60) for j in range(i + 1, 60))
    assert dmin > 0.1, "rotations repeat"

    def index(m):
        k = int(np.argmin(np.abs(flat - m.reshape(9)).max(1)))
        assert np.abs(flat[k] - m.reshape(9)).max() < 1e-12
        return k

    for i in range(60):                   # closure: a group of 60 elements
        for j in range(0, 60, 7):
            index(R[i] @ R[j])
        index(R[i].T)
    V = _icosahedron_vertices()
    for r in R:                           # every element is a symmetry of the solid
        W = V @ r.T
        assert max(np.abs(V - w).max(1).min() for w in W) < 1e-12
    ang = np.round(np.degrees(np.arccos(np.clip((np.einsum("kii->k", R) - 1) / 2, -1, 1))), 3)
    counts = {a: int((ang == a).sum()) for a in np.unique(ang)}
    # 1 identity, 15 half turns (edges), 20 of 120 deg (faces), 12 + 12 of 72/144 deg (vertices)
    assert counts == {0.0: 1, 72.0: 12, 120.0: 20, 144.0: 12, 180.0: 15}


# ------------------------------------------------- inner products, distance --
def test_one_pair_closed_form():
    r, ell = 0.23, 0.2
    p = _problem([[[0.0, 0, 0]], [[r, 0, 0]]], [[0, 1]], ell=ell)
    out = O.distance_and_cosine(p, p["poses0"])
    k = math.exp(-r * r / (2 * ell * ell))
    np.testing.assert_allclose(out["self"], [1.0, 1.0], rtol=1e-15)
    np.testing.assert_allclose(out["cross"], [k], rtol=1e-14)
    np.testing.assert_allclose(out["dist"], [2 - 2 * k], rtol=1e-14)
    np.testing.assert_allclose(out["cos"], [k], rtol=1e-14)
    # d dist / d ell = -2 k r^2 / ell^3
    np.testing.assert_allclose(out["dD_dell"], -2 * k * r * r / ell ** 3, rtol=1e-13)


def test_distance_is_l2_norm_of_smoothed_functions():
    # exp(-|x-y|^2 / 2 ell^2) = (pi ell^2/2)^(-3/2) * integral g(z-x) g(z-y) dz with
    # g(u) = exp(-|u|^2 / ell^2); for points on a line the two transverse
    # integrals give pi ell^2 / 2, the third is done by quadrature.
    rng = np.random.default_rng(5)
    ell = 0.15
    xa = np.zeros((7, 3))
    xb = np.zeros((5, 3))
    xa[:, 0] = rng.uniform(-1, 1, 7)
    xb[:, 0] = rng.uniform(-1, 1, 5)
    p = _problem([xa, xb], [[0, 1]], ell=ell, **ALL)
    d = O.distance_and_cosine(p, p["poses0"])["dist"][0]
    z = np.linspace(-3, 3, 600001)
    f = np.exp(-((z[:, None] - xa[None, :, 0]) ** 2) / ell ** 2).sum(1) \
        - np.exp(-((z[:, None] - xb[None, :, 0]) ** 2) / ell ** 2).sum(1)
    integral = np.trapezoid(f * f, z) * (math.pi * ell ** 2 / 2)
    np.testing.assert_allclose(d, integral / (math.pi * ell ** 2 / 2) ** 1.5, rtol=1e-9)


def test_self_inner_is_the_double_sum_with_labels():
    rng = np.random.default_rng(6)
    x = rng.uniform(0, 0.5, (30, 3))
    sem = rng.dirichlet(np.ones(4), 30).astype(np.float32)
    p = _problem([x, x], [[0, 1]], ell=0.1, sem=[sem, sem])
    got = O.distance_and_cosine(p, p["poses0"])["self"][0]
    rc2 = (3 * 0.1) ** 2
    want = 0.0
    for i in range(30):
        for j in range(30):
            d2 = float(((x[i] - x[j]) ** 2).sum())
            if d2 < rc2:
                want += float(np.dot(sem[i].astype(np.float64), sem[j])) * math.exp(-d2 / (2 * 0.01))
    np.testing.assert_allclose(got, want, rtol=1e-13)


def test_distance_nonnegative_cosine_bounded_zero_for_identical():
    rng = np.random.default_rng(7)
    x = rng.uniform(0, 1, (60, 3))
    sem = rng.dirichlet(np.ones(3), 60).astype(np.float32)
    y = x + rng.normal(scale=0.05, size=x.shape)
    for P in (ALL, {}):
        p = _problem([x, y, x], [[0, 1], [0, 2], [1, 2]], ell=0.15, sem=[sem, sem, sem], **P)
        out = O.distance_and_cosine(p, p["poses0"])
        if P:   # positive definiteness holds for the full sums
            assert (out["dist"] >= -1e-12 * out["self"].max()).all()
            assert (np.abs(out["cos"]) <= 1 + 1e-14).all()
        assert abs(out["dist"][1]) <= 1e-12 * out["self"][0]
        np.testing.assert_allclose(out["cos"][1], 1.0, rtol=1e-14)
    # self terms are pose invariant
    T = np.stack([np.eye(4), O.se3_exp(np.array([0.3, -1, 2, 0.5, 1.0, -2.0])), np.eye(4)])
    p = _problem([x, y, x], [[0, 1]], ell=0.15)
    a = O.distance_and_cosine(p, T)["self"]
    b = O.distance_and_cosine(p, p["poses0"])["self"]
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_ell_derivative_matches_central_differences():
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, (40, 3))
    y = x @ O.se3_exp(np.array([0, 0, 0, 0.05, -0.1, 0.02]))[:3, :3].T + 0.03
    sem = rng.dirichlet(np.ones(3), 40).astype(np.float32)
    p = _problem([x, y], [[0, 1]], ell=0.2, sem=[sem, sem], **ALL)
    T = np.stack([np.eye(4), O.se3_exp(np.array([0.02, 0, -0.01, 0, 0.03, 0]))])
    g = O.distance_and_cosine(p, T)["dD_dell"]
    h = 1e-5

    def D(ell):
        return O.distance_and_cosine(p, T, params=dict(ell=ell))["dist"].sum()

    np.testing.assert_allclose(g, (D(0.2 + h) - D(0.2 - h)) / (2 * h), rtol=1e-6)


def test_ell_step_lowers_the_distance():
    # each outer step multiplies ell by (1 - decay sign(dD/dell)): at the poses
    # a level solved, the summed distance at the next level's ell is lower
    # (every pair kept, so D is smooth in ell and dD/dell is its derivative)
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 2, (150, 3))
    p = _problem([x, x + 0.15], [[0, 1]], ell=0.2, max_iters=20, **ALL)
    out = O.ell_decay_solve(p, decay=0.1, ell_min=0.05, max_outer=3)
    lv = out["levels"]
    assert len(lv) >= 2
    for k in range(len(lv) - 1):
        assert abs(lv[k + 1]["ell"] - max(lv[k]["ell"] * (1 - 0.1 * np.sign(lv[k]["dD_dell"])), 0.05)) < 1e-15
    T = O.lm_solve(p, p["poses0"], params=dict(ell=lv[0]["ell"]))["poses"]
    D0 = O.distance_and_cosine(p, T, params=dict(ell=lv[0]["ell"]))["dist"].sum()
    D1 = O.distance_and_cosine(p, T, params=dict(ell=lv[1]["ell"]))["dist"].sum()
    assert D1 < D0
    # two single points at distance r: D = 2 - 2 exp(-r^2 / 2 ell^2) falls with ell
    two = _problem([[[0.0, 0, 0]], [[0.05, 0, 0]]], [[0, 1]], ell=0.2)
    assert O.distance_and_cosine(two, two["poses0"])["dD_dell"] < 0


# ------------------------------------------------------- rotation search ----
@pytest.mark.parametrize("k", [0, 5, 23, 41, 59])
def test_rotation_search_recovers_a_group_rotation(k):
    rng = np.random.default_rng(9)
    xa = rng.uniform(-1, 1, (120, 3)) * [1.0, 0.6, 0.3]       # anisotropic: no symmetry
    xa = np.vstack([xa, [[0.9, 0.5, 0.2], [0.8, 0.55, 0.25]]])
    R = O.icosahedral_rotations()[k]
    t = np.array([0.4, -0.3, 0.2])
    xb = (xa - t) @ R          # b's points: x_b = R^T (x_a - t), so T_b = [R | t] maps b onto a
    p = _problem([xa, xb], [[0, 1]], ell=0.1)
    cos, best = O.rotation_search(p, 0, 1, p["poses0"])
    assert int(np.argmax(cos)) == k
    np.testing.assert_allclose(cos[k], 1.0, rtol=1e-12)
    assert np.sort(cos)[-2] < 0.9
    np.testing.assert_allclose(best[:3, :3], R, atol=1e-12)
    np.testing.assert_allclose(best[:3, 3], t, atol=1e-12)

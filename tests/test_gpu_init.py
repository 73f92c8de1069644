"""GPU parity of the function-space distance, cosine, d/d ell, the
icosahedral rotation search and the lengthscale-decay loop against the oracle
(Sec. III-A Eq. dist_rkhs, Sec. IV-A, Sec. V-C).

Tolerances: self and cross inner products relative <= 1e-5 (the loss
tolerance: each is one F); the distance and dD/dell are differences of such
sums, so their absolute error is bounded by 1e-5 times the sum of the
magnitudes that enter them; cosines absolute <= 1e-5; poses <= 1e-4 rad / m.
"""
import numpy as np
import pytest

import oracle as O
import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5
POSE_TOL = 1e-4


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01254_gb300 as pk
    pk.load()
    return pk


def _tiny(variant):
    prob = scenes.tiny_problem(seed=41, n_frames=4, n=300, extent=1.0, ell=0.15, color=(variant == "color"))
    if variant == "plain":
        prob["sem"] = None
    if variant == "bf16":
        prob["sem"] = [scenes.round_to_bf16(s) for s in prob["sem"]]
        prob["params"] = dict(prob["params"], sem_bf16=1)
    return prob


def check_inner_products(pk, prob, poses):
    ref = O.distance_and_cosine(prob, poses)
    g = pk.Problem.from_scene(prob)
    try:
        out = g.inner_products(poses)
        again = g.inner_products(poses)          # cached self terms, same result
    finally:
        g.close()
    for k in ("self", "cross", "dist", "cos"):
        assert np.array_equal(out[k], again[k])
    np.testing.assert_allclose(out["self"], ref["self"], rtol=TOL)
    np.testing.assert_allclose(out["cross"], ref["cross"], rtol=TOL, atol=TOL * ref["self"].max())
    edges = np.asarray(prob["edges"]).reshape(-1, 2)
    scale = ref["self"][edges[:, 0]] + ref["self"][edges[:, 1]]
    assert (np.abs(out["dist"] - ref["dist"]) <= TOL * scale).all(), (out["dist"], ref["dist"])
    np.testing.assert_allclose(out["cos"], ref["cos"], atol=TOL)
    P = dict(O.DEFAULTS)
    P.update(prob["params"])
    mag = P["sigma"] ** 2 / P["ell"] ** 3 * (ref["self_E"][edges].sum() + 2 * ref["cross_E"].sum())
    assert abs(out["dD_dell"] - ref["dD_dell"]) <= TOL * mag, (out["dD_dell"], ref["dD_dell"])
    return out, ref


@pytest.mark.parametrize("variant", ["plain", "fp32", "bf16", "color"])
def test_inner_products_parity(pk, variant):
    prob = _tiny(variant)
    check_inner_products(pk, prob, prob["poses0"])


def test_inner_products_identical_frames_and_empty_frame(pk):
    prob = scenes.tiny_problem(seed=42, n_frames=3, n=400, extent=1.0, ell=0.15)
    prob["xyz"][1] = prob["xyz"][0].copy()
    prob["sem"][1] = prob["sem"][0].copy()
    prob["xyz"][2] = prob["xyz"][2][:0]
    prob["sem"][2] = prob["sem"][2][:0]
    poses = np.stack([np.eye(4)] * 3)
    out, ref = check_inner_products(pk, prob, poses)
    assert abs(out["cos"][0] - 1.0) <= TOL                   # edge (0, 1): identical clouds
    assert abs(out["dist"][0]) <= TOL * 2 * out["self"][0]
    assert out["self"][2] == 0.0 and out["cos"][1] == 0.0    # empty frame


def test_inner_products_lidar_reduced(pk):
    prob = scenes.lidar_street_problem(seed=43, n_frames=3, n_points=3000)
    check_inner_products(pk, prob, prob["poses0"])


# ------------------------------------------------------- rotation search ----
def _match(Rg, Ro):
    """index into Ro of every rotation of Rg (the same set, any order)."""
    idx = []
    for r in Rg:
        d = np.abs(Ro - r).reshape(len(Ro), -1).max(1)
        j = int(np.argmin(d))
        assert d[j] < 1e-9
        idx.append(j)
    assert sorted(idx) == list(range(len(Ro)))
    return np.array(idx)


def test_rotation_table_is_the_oracles_group(pk):
    prob = scenes.object_pair_problem(seed=3, n=300)
    g = pk.Problem.from_scene(prob)
    try:
        out = g.rotation_search(0, 1, prob["poses0"])
    finally:
        g.close()
    _match(out["rotations"], O.icosahedral_rotations())
    ang = np.degrees(np.arccos(np.clip((np.einsum("kii->k", out["rotations"]) - 1) / 2, -1, 1)))
    # the paper's listing order: identity, 15 half turns, 20 third turns, 24 fifth turns
    assert ang[0] < 1e-6 and (np.abs(ang[1:16] - 180) < 1e-3).all()
    assert (np.abs(ang[16:36] - 120) < 1e-3).all()
    assert (np.minimum(np.abs(ang[36:] - 72), np.abs(ang[36:] - 144)) < 1e-3).all()


@pytest.mark.parametrize("labels", [False, True])
def test_rotation_search_parity(pk, labels):
    prob = scenes.object_pair_problem(seed=5, angle_deg=120.0, n=800, outlier_ratio=0.125, crop_ratio=0.125,
                                      ell=0.1, labels=labels)
    poses = np.stack([scenes.random_pose(np.random.default_rng(1), 30, 0.2), np.eye(4)])
    cos_o, best_o = O.rotation_search(prob, 0, 1, poses)
    g = pk.Problem.from_scene(prob)
    try:
        out = g.rotation_search(0, 1, poses)
    finally:
        g.close()
    idx = _match(out["rotations"], O.icosahedral_rotations())
    np.testing.assert_allclose(out["cos"], cos_o[idx], atol=TOL)
    top = np.sort(cos_o)
    if top[-1] - top[-2] > 1e-4:
        assert idx[out["best"]] == int(np.argmax(cos_o))
        dr, dt = O.pose_error(out["best_pose"], best_o)
        assert dr <= 1e-9 and dt <= 1e-9


@pytest.mark.parametrize("k", [0, 7, 20, 44])
def test_rotation_search_recovers_a_group_rotation(pk, k):
    rng = np.random.default_rng(11)
    xa = rng.uniform(-1, 1, (3000, 3)) * [1.0, 0.6, 0.3]
    xa = np.vstack([xa, rng.normal(size=(300, 3)) * 0.05 + [0.9, 0.5, 0.2]])
    g0 = pk.Problem(xyz=[xa, xa], edges=[[0, 1]], ell=0.1)
    try:
        R = g0.rotation_search(0, 1, np.stack([np.eye(4)] * 2))["rotations"][k]
    finally:
        g0.close()
    t = np.array([0.4, -0.3, 0.2])
    xb = (xa - t) @ R
    g = pk.Problem(xyz=[xa, xb], edges=[[0, 1]], ell=0.1)
    try:
        out = g.rotation_search(0, 1, np.stack([np.eye(4)] * 2))
    finally:
        g.close()
    assert out["best"] == k
    assert abs(out["cos"][k] - 1.0) <= TOL
    dr, dt = O.pose_error(out["best_pose"], scenes.make_pose(R, t))
    assert dr <= 1e-9 and dt <= 1e-9


def test_rotation_search_rejects_bad_frames(pk):
    prob = scenes.object_pair_problem(seed=3, n=300)
    g = pk.Problem.from_scene(prob)
    try:
        for a, b in ((0, 0), (0, 2), (-1, 1)):
            with pytest.raises(pk.RkhsbaError):
                g.rotation_search(a, b, prob["poses0"])
    finally:
        g.close()


@pytest.mark.parametrize("angle", [90.0, 180.0])
def test_global_initialisation_protocol(pk, angle):
    """Two noisy, cropped scans under a 90 / 180 degree rotation about a
    random axis and a 0.5 translation: rotation search, then the LM solve at
    ell = 0.1, 0.05, 0.03, recovers the relative pose."""
    errs = []
    for seed in range(4):
        prob = scenes.object_pair_problem(seed=200 + seed, angle_deg=angle, n=4000, outlier_ratio=0.125,
                                          crop_ratio=0.125, ell=0.1, labels=True)
        g = pk.Problem.from_scene(prob)
        try:
            T = np.stack([np.eye(4), g.rotation_search(0, 1, prob["poses0"])["best_pose"]])
        finally:
            g.close()
        for ell in (0.1, 0.05, 0.03):
            g = pk.Problem.from_scene(prob, ell=ell, max_iters=40)
            try:
                T, _ = g.solve(T)
            finally:
                g.close()
        errs.append(O.pose_error(T[1], prob["poses_gt"][1]))
    errs = np.array(errs)
    print("angle", angle, "rotation / translation errors", errs.round(4).tolist())
    assert (errs[:, 0] < 0.05).sum() >= 3, errs
    assert np.median(errs[:, 0]) < 0.03, errs


# ------------------------------------------------------- lengthscale decay --
def test_ell_decay_parity(pk):
    prob = scenes.tiny_problem(seed=45, n_frames=3, n=300, extent=1.0, ell=0.2)
    prob["params"] = dict(prob["params"], max_iters=30)
    ref = O.ell_decay_solve(prob, params=dict(max_iters=30), decay=0.2, ell_min=0.05, max_outer=4)
    g = pk.Problem.from_scene(prob)
    try:
        T, info = g.solve_ell_decay(prob["poses0"], decay=0.2, ell_min=0.05, max_outer=4)
    finally:
        g.close()
    assert info["levels"] == len(ref["levels"])
    np.testing.assert_array_equal(info["ell"], [lv["ell"] for lv in ref["levels"]])
    assert np.all(np.sign(info["dD_dell"]) == np.sign([lv["dD_dell"] for lv in ref["levels"]]))
    dr = max(O.pose_error(a, b)[0] for a, b in zip(T, ref["poses"]))
    dt = max(O.pose_error(a, b)[1] for a, b in zip(T, ref["poses"]))
    assert dr <= POSE_TOL and dt <= POSE_TOL, (dr, dt)


def test_ell_decay_rejects_bad_schedule(pk):
    prob = scenes.tiny_problem(seed=46, n_frames=2, n=100)
    g = pk.Problem.from_scene(prob)
    try:
        for kw in (dict(decay=0.0), dict(decay=1.5), dict(max_outer=0), dict(ell_min=-1.0)):
            with pytest.raises(pk.RkhsbaError):
                g.solve_ell_decay(prob["poses0"], **kw)
    finally:
        g.close()


# ------------------------------------------------- full-size, sampled --------
def test_inner_products_full_size_sampled(pk):
    """Bench workload (8 x 20k LiDAR points, 28 edges): the GPU's values for
    two sampled edges and their frames' self terms against the oracle."""
    prob = scenes.lidar_street_problem(seed=1434)
    g = pk.Problem.from_scene(prob)
    try:
        out = g.inner_products(prob["poses0"])
    finally:
        g.close()
    edges = np.asarray(prob["edges"])
    for e in (0, 17):
        a, b = (int(v) for v in edges[e])
        sub = dict(prob, xyz=[prob["xyz"][a], prob["xyz"][b]], sem=[prob["sem"][a], prob["sem"][b]],
                   edges=np.array([[0, 1]], np.int32))
        ref = O.distance_and_cosine(sub, prob["poses0"][[a, b]])
        np.testing.assert_allclose(out["self"][[a, b]], ref["self"], rtol=TOL)
        np.testing.assert_allclose(out["cross"][e], ref["cross"][0], rtol=TOL)
        np.testing.assert_allclose(out["cos"][e], ref["cos"][0], atol=TOL)


def test_rotation_search_full_size_sampled(pk):
    """8000-point scans (the largest size of the paper's timing study): the
    cosines of sampled candidates against the oracle's inner products
    at those candidate poses (three sampled, the best among them)."""
    prob = scenes.object_pair_problem(seed=210, angle_deg=180.0, n=8000, outlier_ratio=0.125, crop_ratio=0.125,
                                      ell=0.1, labels=True)
    g = pk.Problem.from_scene(prob)
    try:
        out = g.rotation_search(0, 1, prob["poses0"])
    finally:
        g.close()
    xa, xb = prob["xyz"]
    sa, sb = prob["sem"]
    P = dict(O.DEFAULTS)
    P.update(prob["params"])
    Sa = O.self_inner(xa, sa, None, P)
    Sb = O.self_inner(xb, sb, None, P)
    mua, mub = xa.mean(0), xb.mean(0)
    for k in sorted({0, 29, int(out["best"])}):
        R = out["rotations"][k]
        Tb = np.eye(4)
        Tb[:3, :3] = R
        Tb[:3, 3] = mua - R @ mub
        cos = O.inner_product(xa, xb, np.eye(4), Tb, sa, sb, None, None, P) / np.sqrt(Sa * Sb)
        assert abs(out["cos"][k] - cos) <= TOL, (k, out["cos"][k], cos)

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated by the precision contract of the workloads and, for H,
derived from FP32 per-query accumulation of moments about the frame origin):
  loss            relative error            <= 1e-5
  gradient        relative 2-norm error     <= 1e-4
  Gauss-Newton H  relative Frobenius error  <= 1e-4
  converged poses                           <= 1e-4 rad and 1e-4 m
  pair sets       bit-exact outside |(|d| - r_c)| <= 1e-6 r_c
"""
import numpy as np
import pytest

import oracle as O
import scenes

pytestmark = pytest.mark.gpu

LOSS_TOL, GRAD_TOL, H_TOL, POSE_TOL = 1e-5, 1e-4, 1e-4, 1e-4


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01254_gb300 as pk
    pk.load()
    return pk


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _reln(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _band_pairs(prob, poses, e):
    """Oracle pairs whose |d| lies within 1e-6 r_c of the cutoff (either side)."""
    P = dict(O.DEFAULTS)
    P.update(prob["params"])
    rc = P["cutoff_mult"] * P["ell"]
    a, b = (int(v) for v in prob["edges"][e])
    pa = np.asarray(prob["xyz"][a], np.float64) @ poses[a][:3, :3].T + poses[a][:3, 3]
    pb = np.asarray(prob["xyz"][b], np.float64) @ poses[b][:3, :3].T + poses[b][:3, 3]
    i, j = O.pairs_kdtree(pa, pb, rc * (1 + 2e-6))
    d = np.linalg.norm(pa[i] - pb[j], axis=1)
    m = np.abs(d - rc) <= 1e-6 * rc
    return set(zip(i[m].tolist(), j[m].tolist()))


def check_eval(pk, prob, poses, edge_subset=None, n_band_max=None, uq=None):
    sub = prob if edge_subset is None else dict(prob, edges=np.asarray(prob["edges"])[edge_subset])
    ref = O.evaluate(sub, poses)
    g = pk.Problem.from_scene(sub)
    try:
        if uq:
            g.set_tuning(uq, 0)
        out = g.eval(poses, want_H=True, want_blocks=True)
    finally:
        g.close()
    assert ref["n_pairs"] > 0
    # pair counts agree up to pairs in the cutoff band
    diff = np.abs(out["edge_pairs"] - ref["edge_pairs"])
    assert diff.sum() <= max(3, 1e-6 * ref["n_pairs"]), (out["edge_pairs"], ref["edge_pairs"])
    assert _rel(out["loss"], ref["loss"]) <= LOSS_TOL, (out["loss"], ref["loss"])
    assert _reln(out["grad"], ref["grad"]) <= GRAD_TOL, _reln(out["grad"], ref["grad"])
    assert _reln(out["H"], ref["H"]) <= H_TOL, _reln(out["H"], ref["H"])
    for e in range(len(sub["edges"])):
        if ref["edge_pairs"][e] > 0:
            assert _reln(out["H_blocks"][e], ref["H_blocks"][e]) <= H_TOL
    return out, ref


# ------------------------------------------------------------ small cases ---
@pytest.mark.parametrize("variant", ["plain", "fp32", "bf16", "color"])
def test_tiny_eval_parity(pk, variant):
    prob = scenes.tiny_problem(seed=31, n_frames=4, n=300, extent=1.0, ell=0.15,
                               color=(variant == "color"))
    if variant == "plain":
        prob["sem"] = None
    if variant == "bf16":
        prob["sem"] = [scenes.round_to_bf16(s) for s in prob["sem"]]
        prob["params"] = dict(prob["params"], sem_bf16=1)
    check_eval(pk, prob, prob["poses0"])


@pytest.mark.parametrize("bf16,uq", [(0, None), (1, 64)])
def test_ragged_sizes_and_many_tiles(pk, bf16, uq):
    prob = scenes.tiny_problem(seed=32, n_frames=3, n=777, extent=2.5, ell=0.1)
    prob["xyz"][1] = prob["xyz"][1][:531]
    prob["sem"][1] = prob["sem"][1][:531]
    prob["xyz"][2] = prob["xyz"][2][:1]
    prob["sem"][2] = prob["sem"][2][:1]
    if bf16:
        prob["sem"] = [scenes.round_to_bf16(s) for s in prob["sem"]]
        prob["params"] = dict(prob["params"], sem_bf16=1)
    check_eval(pk, prob, prob["poses0"], uq=uq)


def test_pair_sets_bit_exact_outside_band(pk):
    for prob in (scenes.tiny_problem(seed=33, n_frames=2, n=400, extent=1.2, ell=0.12),
                 scenes.config_problem(1)):
        T = prob["poses0"]
        g = pk.Problem.from_scene(prob)
        try:
            gi, gj, n = g.edge_pairs(T, 0)
        finally:
            g.close()
        ri, rj = O.edge_pairs(prob, T, 0)
        band = _band_pairs(prob, T, 0)
        gs = set(zip(gi.tolist(), gj.tolist())) - band
        rs = set(zip(ri.tolist(), rj.tolist())) - band
        assert n == len(gi)
        assert len(gs) == len(set(zip(gi.tolist(), gj.tolist())) - band)
        assert gs == rs


def test_plane_sphere_eval_parity(pk):
    prob = scenes.config_problem(1)
    for T in (prob["poses0"], prob["poses_gt"]):
        check_eval(pk, prob, T)


def test_lidar_reduced_eval_parity(pk):
    prob = scenes.lidar_street_problem(seed=41, n_frames=4, n_points=4000)
    check_eval(pk, prob, prob["poses0"])
    check_eval(pk, prob, prob["poses_gt"])


def test_window_bf16_reduced_eval_parity(pk):
    prob = scenes.window_problem(seed=42, window=3, n_points=6000)
    check_eval(pk, prob, prob["poses0"])


@pytest.mark.slow
def test_lidar_full_size_sampled_edges(pk):
    """The 8 x 20k LiDAR workload at full size; the oracle checks 3 of the 28
    edges (first, middle, last) through a problem holding only those edges."""
    prob = scenes.config_problem(2)
    check_eval(pk, prob, prob["poses0"], edge_subset=[0, 13, 27])


def test_full_size_gauge_invariance(pk):
    prob = scenes.config_problem(2)
    g = pk.Problem.from_scene(prob)
    try:
        T = prob["poses0"]
        a = g.eval(T, want_H=False)
        G = scenes.random_pose(np.random.default_rng(5), 30.0, 3.0)
        b = g.eval(np.stack([G @ t for t in T]), want_H=False)
        # a common left motion moves every query by a rigid motion of frame a:
        # the pair set and F can only change through FP32 rounding at the band
        assert _rel(b["loss"], a["loss"]) <= 1e-5
    finally:
        g.close()


# --------------------------------------------------------------- edge cases -
@pytest.mark.parametrize("bf16,uq", [(0, None), (1, 32), (1, 64), (1, 7)])
def test_degenerate_inputs(pk, bf16, uq):
    # one cell holding 500 points (home cells of many full units), an empty
    # frame, a far frame; FP32 labels and BF16 labels at several unit sizes
    rng = np.random.default_rng(7)
    blob = np.full((500, 3), 0.25) + rng.normal(scale=1e-4, size=(500, 3))   # one cell
    far = rng.uniform(100, 101, size=(50, 3))
    lab = scenes.dirichlet_labels(rng, rng.integers(0, 4, 500), 4)
    if bf16:
        lab = scenes.round_to_bf16(lab)
    prob = dict(xyz=[blob, blob[:200] + 0.01, np.zeros((0, 3)), far],
                sem=[lab, lab[:200], np.zeros((0, 4), np.float32), lab[:50]], rgb=None,
                edges=np.array([[0, 1], [1, 2], [0, 3], [2, 3]], np.int32),
                params=dict(ell=0.1, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_bf16=bf16))
    T = np.stack([np.eye(4)] * 4)
    out, ref = check_eval(pk, prob, T, uq=uq)
    assert out["edge_pairs"][1] == 0 and out["edge_pairs"][2] == 0 and out["edge_pairs"][3] == 0


def test_no_pairs_anywhere(pk):
    prob = dict(xyz=[np.zeros((10, 3)), np.full((10, 3), 50.0)], sem=None, rgb=None,
                edges=np.array([[0, 1]], np.int32), params=dict(ell=0.1))
    g = pk.Problem.from_scene(prob)
    try:
        out = g.eval(np.stack([np.eye(4)] * 2))
    finally:
        g.close()
    assert out["n_pairs"] == 0 and out["loss"] == 0.0
    assert not out["grad"].any() and not out["H"].any()


def test_invalid_inputs_are_rejected(pk):
    ok = scenes.tiny_problem(seed=8, n_frames=2, n=20)
    bad = [dict(ok, xyz=[ok["xyz"][0].copy(), ok["xyz"][1].copy()]) for _ in range(4)]
    bad[0]["xyz"][0][3, 1] = np.nan
    bad[1]["edges"] = np.array([[0, 0]], np.int32)
    bad[2]["edges"] = np.array([[0, 1], [1, 0]], np.int32)
    bad[3]["edges"] = np.array([[0, 2]], np.int32)
    for prob in bad:
        with pytest.raises(pk.RkhsbaError) as ei:
            pk.Problem.from_scene(prob)
        assert ei.value.status == 1
    g = pk.Problem.from_scene(ok)
    try:
        T = np.stack([np.eye(4)] * 2)
        T[1, 0, 0] = 1.1
        with pytest.raises(pk.RkhsbaError):
            g.eval(T)
    finally:
        g.close()
    with pytest.raises(pk.RkhsbaError):
        pk.Problem(ok["xyz"], [np.zeros((20, 40), np.float32)] * 2, None, ok["edges"], ell=0.1)


def test_evaluation_is_bit_reproducible(pk):
    prob = scenes.lidar_street_problem(seed=43, n_frames=3, n_points=3000)
    g = pk.Problem.from_scene(prob)
    try:
        a = g.eval(prob["poses0"])
        b = g.eval(prob["poses0"])
    finally:
        g.close()
    g2 = pk.Problem.from_scene(prob)
    try:
        c = g2.eval(prob["poses0"])
    finally:
        g2.close()
    for r in (b, c):
        assert r["loss"] == a["loss"]
        assert np.array_equal(r["grad"], a["grad"]) and np.array_equal(r["H"], a["H"])


# -------------------------------------------------------------------- solve -
def _pose_errs(Ta, Tb):
    return max(O.pose_error(a, b)[0] for a, b in zip(Ta, Tb)), \
        max(O.pose_error(a, b)[1] for a, b in zip(Ta, Tb))


def test_solve_parity_plane_sphere(pk):
    prob = scenes.config_problem(1)
    rng = np.random.default_rng(9)
    init = np.stack([prob["poses_gt"][0], scenes.perturb(rng, prob["poses_gt"][1], 2.0, 0.05)])
    ref = O.lm_solve(prob, poses0=init, params=dict(max_iters=100))
    g = pk.Problem.from_scene(prob, max_iters=100)
    try:
        T, info = g.solve(init)
    finally:
        g.close()
    dr, dt = _pose_errs(T, ref["poses"])
    assert dr <= POSE_TOL and dt <= POSE_TOL, (dr, dt, info, ref["status"], ref["iters"])
    assert info["status"] == "OK"


def test_solve_parity_window_bf16(pk):
    prob = scenes.window_problem(seed=44, window=3, n_points=3000)
    ref = O.lm_solve(prob, params=dict(max_iters=60))
    g = pk.Problem.from_scene(prob, max_iters=60)
    try:
        T, info = g.solve(prob["poses0"])
    finally:
        g.close()
    dr, dt = _pose_errs(T, ref["poses"])
    assert dr <= POSE_TOL and dt <= POSE_TOL, (dr, dt, info, ref["status"], ref["iters"])


def test_solve_recovers_ground_truth_on_identical_clouds(pk):
    prob = scenes.plane_sphere_problem(seed=15, n=1500, same_points=True, angle_deg=2.0,
                                       trans=0.04, ell=0.1)
    g = pk.Problem.from_scene(prob, max_iters=80)
    try:
        T, info = g.solve(prob["poses0"])
    finally:
        g.close()
    dr, dt = O.pose_error(T[1], prob["poses_gt"][1])
    assert dr < 1e-5 and dt < 1e-5, (dr, dt, info)


# ------------------------------------------------ every label width -----------
@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("sem_dim", [1, 5, 9, 13, 17, 21, 25, 32])
def test_every_label_width(pk, sem_dim, bf16):
    """Each padded label width of the pair kernel (FP32 rows of 4..32 floats,
    BF16 rows of 8..32 values on the tensor-core Gram path, one or two k16
    steps) against the oracle, with and without the top-k variant."""
    rng = np.random.default_rng(sem_dim)
    prob = scenes.tiny_problem(seed=80 + sem_dim, n_frames=3, n=300, extent=1.0, ell=0.15)
    lab = [rng.dirichlet(np.ones(sem_dim), len(x)).astype(np.float32) for x in prob["xyz"]]
    if bf16:
        lab = [scenes.round_to_bf16(s) for s in lab]
    prob["sem"] = lab
    prob["params"] = dict(prob["params"], sem_bf16=int(bf16))
    check_eval(pk, prob, prob["poses0"])
    prob["params"] = dict(prob["params"], top_k=5)
    check_eval(pk, prob, prob["poses0"])


def test_many_frames(pk):
    """4096 frames (the frame limit) of 12 points on a chain of 4095 edges:
    loss and gradient against the oracle's per-edge sums (the 6K x 6K matrix
    is not formed on the host)."""
    rng = np.random.default_rng(4096)
    K, n = 4096, 12
    base = rng.uniform(0, 0.4, (n, 3))
    xyz = [base + rng.normal(scale=0.02, size=base.shape) for _ in range(K)]
    edges = np.array([[m, m + 1] for m in range(K - 1)], np.int32)
    poses = np.stack([scenes.random_pose(rng, 1.0, 0.01) for _ in range(K)])
    poses[0] = np.eye(4)
    prob = dict(xyz=xyz, sem=None, rgb=None, edges=edges, poses0=poses,
                params=dict(ell=0.1, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_bf16=0))
    g = pk.Problem.from_scene(prob)
    try:
        out = g.eval(poses, want_H=False)
    finally:
        g.close()
    F = 0.0
    b = np.zeros(6 * K)
    for a, c in edges:
        t = O.edge_terms(xyz[a], xyz[c], poses[a], poses[c], params=prob["params"])
        F += t["F"]
        b[6 * a:6 * a + 6] += t["b"][:6]
        b[6 * c:6 * c + 6] += t["b"][6:]
    grad = b / 0.1 ** 2
    assert abs(out["loss"] + F) <= LOSS_TOL * F
    assert _reln(out["grad"], grad) <= GRAD_TOL


def test_solve_parity_large_system(pk):
    """40 frames: the 234 x 234 damped system is factored by the blocked
    multi-block Cholesky (n >= 192); poses after 10 LM iterations against the
    oracle's LM."""
    rng = np.random.default_rng(4040)
    K, n = 40, 150
    base = rng.uniform(0, 0.6, (n, 3))
    gt = [np.eye(4)] + [scenes.random_pose(rng, 10.0, 0.1) for _ in range(K - 1)]
    xyz = [scenes.to_local(base + rng.normal(scale=0.01, size=base.shape), T) for T in gt]
    init = np.stack([gt[0]] + [scenes.perturb(rng, T, 2.0, 0.03) for T in gt[1:]])
    edges = np.array([[m, m + d] for m in range(K) for d in (1, 2) if m + d < K], np.int32)
    prob = dict(xyz=xyz, sem=None, rgb=None, edges=edges, poses0=init,
                params=dict(ell=0.1, cutoff_mult=3.0, sigma=1.0, ell_color=0.0, sem_bf16=0))
    ref = O.lm_solve(prob, params=dict(max_iters=10))
    g = pk.Problem.from_scene(prob, max_iters=10)
    try:
        T, info = g.solve(init)
    finally:
        g.close()
    assert info["iters"] == ref["iters"]
    dr, dt = _pose_errs(T, ref["poses"])
    assert dr <= POSE_TOL and dt <= POSE_TOL, (dr, dt, info, ref["status"])
    moved = max(O.pose_error(a, b)[1] for a, b in zip(ref["poses"], init))
    assert moved > 100 * POSE_TOL


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("label_scale,ell", [(1e3, 0.15), (1e-3, 0.15), (1.0, 40.0), (1.0, 0.002)])
def test_dense_kernel_scaling_extremes(pk, bf16, label_scale, ell):
    """The dense kernel carries weights, features and (FP32) label parts in
    FP16 under power-of-two scales chosen from the label norms and the cell
    size; labels far from unit norm and lengthscales far from the workloads'
    must still match the oracle."""
    prob = scenes.tiny_problem(seed=91, n_frames=3, n=300, extent=1.0, ell=0.15)
    geo = ell / 0.15
    prob["xyz"] = [x * geo for x in prob["xyz"]]
    prob["poses0"] = prob["poses0"].copy()
    prob["poses0"][:, :3, 3] *= geo
    lab = [np.asarray(s, np.float32) * np.float32(label_scale) for s in prob["sem"]]
    if bf16:
        lab = [scenes.round_to_bf16(s) for s in lab]
    prob["sem"] = lab
    prob["params"] = dict(prob["params"], ell=ell, sem_bf16=int(bf16))
    check_eval(pk, prob, prob["poses0"])

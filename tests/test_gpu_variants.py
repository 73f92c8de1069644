"""GPU parity of the sparse-sum variants against the oracle: semantic pruning
(pairs with <l_i, l_j> < sem_min dropped, Sec. VII) and the top-k neighbour
limit (per point of an edge's second frame, the k pairs of largest w; the
8-neighbour setting of Sec. VI, time analysis).

Tolerances as for the full sum (loss 1e-5 relative, gradient and H 1e-4
relative norm, poses 1e-4).  The kept pair counts may differ by pairs whose
label product or weight sits within FP32 rounding of the threshold or of the
k-th largest weight; such pairs are few and carry matching weights.
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


def _reln(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def check(pk, prob, poses, max_pair_diff=3):
    ref = O.evaluate(prob, poses)
    g = pk.Problem.from_scene(prob)
    try:
        out = g.eval(poses, want_H=True)
    finally:
        g.close()
    assert ref["n_pairs"] > 0
    assert abs(int(out["n_pairs"]) - int(ref["n_pairs"])) <= max_pair_diff, (out["n_pairs"], ref["n_pairs"])
    assert abs(out["loss"] - ref["loss"]) <= LOSS_TOL * abs(ref["loss"]), (out["loss"], ref["loss"])
    assert _reln(out["grad"], ref["grad"]) <= GRAD_TOL
    assert _reln(out["H"], ref["H"]) <= H_TOL
    return out, ref


@pytest.mark.parametrize("variant", ["fp32", "bf16", "color"])
@pytest.mark.parametrize("top_k", [1, 3, 8])
def test_top_k_parity(pk, variant, top_k):
    prob = scenes.tiny_problem(seed=71, n_frames=3, n=400, extent=1.0, ell=0.15, color=(variant == "color"))
    if variant == "bf16":
        prob["sem"] = [scenes.round_to_bf16(s) for s in prob["sem"]]
        prob["params"] = dict(prob["params"], sem_bf16=1)
    prob["params"] = dict(prob["params"], top_k=top_k)
    out, ref = check(pk, prob, prob["poses0"])
    full = O.evaluate(dict(prob, params=dict(prob["params"], top_k=0)), prob["poses0"])
    assert ref["n_pairs"] < full["n_pairs"]


def test_top_k_without_labels(pk):
    prob = scenes.tiny_problem(seed=72, n_frames=3, n=500, extent=1.5, ell=0.12)
    prob["sem"] = None
    prob["params"] = dict(prob["params"], top_k=8)
    check(pk, prob, prob["poses0"])


@pytest.mark.parametrize("sem_min", [0.05, 0.2, 0.5])
def test_semantic_pruning_parity(pk, sem_min):
    prob = scenes.tiny_problem(seed=73, n_frames=3, n=400, extent=1.0, ell=0.15)
    prob["params"] = dict(prob["params"], sem_min=sem_min)
    out, ref = check(pk, prob, prob["poses0"])
    full = O.evaluate(dict(prob, params=dict(prob["params"], sem_min=0.0)), prob["poses0"])
    assert ref["n_pairs"] < full["n_pairs"]


def test_top_8_lidar_reduced(pk):
    prob = scenes.lidar_street_problem(seed=74, n_frames=3, n_points=4000)
    prob["params"] = dict(prob["params"], top_k=8, sem_min=0.1)
    check(pk, prob, prob["poses0"], max_pair_diff=20)


def test_top_k_solve_parity(pk):
    prob = scenes.tiny_problem(seed=75, n_frames=3, n=300, extent=1.0, ell=0.15)
    prob["params"] = dict(prob["params"], top_k=4, max_iters=40)
    ref = O.lm_solve(prob, params=dict(max_iters=40))
    g = pk.Problem.from_scene(prob)
    try:
        T, info = g.solve(prob["poses0"])
    finally:
        g.close()
    dr = max(O.pose_error(a, b)[0] for a, b in zip(T, ref["poses"]))
    dt = max(O.pose_error(a, b)[1] for a, b in zip(T, ref["poses"]))
    assert dr <= POSE_TOL and dt <= POSE_TOL, (dr, dt, info)


def test_variant_parameters_are_checked(pk):
    prob = scenes.tiny_problem(seed=76, n_frames=2, n=50)
    for over in (dict(top_k=9), dict(top_k=-1), dict(sem_min=-0.5), dict(sem_min=float("nan"))):
        with pytest.raises(pk.RkhsbaError) as ei:
            pk.Problem.from_scene(prob, **over)
        assert ei.value.status == 1

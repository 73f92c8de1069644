"""GPU parity at the workloads' stated sizes, on sampled edges.

The small parity cases never reach some paths of the pair kernel that the
full workloads take: hundreds of candidates per query, home cells holding
several 32-query units, fixed-point scales built from 1e5 x 1e5 point
bounds, hundreds of edges in one launch, the 384 x 384 LM system.  Here the
CUDA path runs the full problems; the FP64 oracle recomputes sampled edges at
full density (its sums split over slices of frame b's points and spread over
the host cores, oracle.split_sum):

  * mapping 64 x 100k (BF16 labels, 516 edges with loop closures), with units
    of 32 and of 64 queries: the whole problem is evaluated in one pass (the
    bench's launch configuration) and
    its per-edge 12 x 12 blocks and pair counts for the sampled edges must
    equal, bit for bit, those of a problem holding only the sampled edges,
    which is compared with the oracle (loss, gradient, H, blocks);
  * window 10 x 50k (BF16 labels, 10% outliers): the same on sampled edges;
  * LiDAR registration (8 x 20k geometry at 3 frames x 5000 points, the
    config's 15 deg / 0.5 m perturbations): the LM solve's poses after a fixed
    number of iterations against the oracle's LM.

Tolerances as in test_gpu_parity: loss 1e-5 relative, gradient 1e-4 relative
2-norm, H and every block 1e-4 relative Frobenius, poses 1e-4 rad / 1e-4 m;
pair counts equal up to pairs within 1e-6 r_c of the cutoff.
"""
import numpy as np
import pytest

import oracle as O
import scenes
from oracle.split_sum import evaluate_split

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


_REF = {}


def _sampled_edge_parity(pk, prob, ids, full_blocks=None, full_pairs=None, uq=None, key=None):
    T = prob["poses0"]
    sub = dict(prob, edges=np.asarray(prob["edges"])[ids])
    g = pk.Problem.from_scene(sub)
    try:
        if uq:
            g.set_tuning(uq, 0)
        out = g.eval(T, want_H=True, want_blocks=True)
    finally:
        g.close()
    if full_blocks is not None:
        for k, e in enumerate(ids):
            assert np.array_equal(out["H_blocks"][k], full_blocks[e]), "edge %d depends on the other edges" % e
            assert out["edge_pairs"][k] == full_pairs[e]
    if key is None or key not in _REF:
        ref = evaluate_split(prob, T, ids)
        if key is not None:
            _REF[key] = ref
    ref = _REF[key] if key is not None else ref
    assert ref["n_pairs"] > 0
    diff = np.abs(out["edge_pairs"] - ref["edge_pairs"])
    assert diff.sum() <= max(3, 1e-6 * ref["n_pairs"]), (out["edge_pairs"], ref["edge_pairs"])
    assert abs(out["loss"] - ref["loss"]) <= LOSS_TOL * abs(ref["loss"]), (out["loss"], ref["loss"])
    assert _reln(out["grad"], ref["grad"]) <= GRAD_TOL, _reln(out["grad"], ref["grad"])
    assert _reln(out["H"], ref["H"]) <= H_TOL, _reln(out["H"], ref["H"])
    for k in range(len(ids)):
        assert _reln(out["H_blocks"][k], ref["H_blocks"][k]) <= H_TOL, (ids[k], _reln(out["H_blocks"][k],
                                                                                     ref["H_blocks"][k]))
    return out, ref


@pytest.mark.parametrize("uq", [32, 64])
def test_mapping_64x100000_sampled_edges(pk, uq):
    # units of 32 queries (default) and of 64 (the setting the autotuner
    # picks for this workload in the bench)
    prob = scenes.config_problem(5)
    E = np.asarray(prob["edges"])
    assert len(prob["xyz"]) == 64 and len(E) == 516
    near = int(np.nonzero((E[:, 0] == 30) & (E[:, 1] == 37))[0][0])
    closure = int(np.nonzero(E[:, 1] - E[:, 0] > 7)[0][0])          # first loop-closure edge
    ids = [0, near, closure]
    g = pk.Problem.from_scene(prob)
    try:
        g.set_tuning(uq, 0)
        full = g.eval(prob["poses0"], want_H=False, want_blocks=True)
    finally:
        g.close()
    assert full["n_pairs"] > 1e10
    out, ref = _sampled_edge_parity(pk, prob, ids, full["H_blocks"], full["edge_pairs"], uq=uq, key="mapping")
    # dense: hundreds of candidates inside r_c per query of the sampled edges
    assert ref["n_pairs"] / sum(len(prob["xyz"][int(E[e, 1])]) for e in ids) > 200


def test_window_10x50000_sampled_edges(pk):
    prob = scenes.config_problem(3, window=10)
    E = np.asarray(prob["edges"])
    assert len(E) == 45
    ids = [0, int(np.nonzero((E[:, 0] == 4) & (E[:, 1] == 7))[0][0]),
           int(np.nonzero((E[:, 0] == 0) & (E[:, 1] == 9))[0][0])]
    g = pk.Problem.from_scene(prob)
    try:
        full = g.eval(prob["poses0"], want_H=False, want_blocks=True)
    finally:
        g.close()
    _sampled_edge_parity(pk, prob, ids, full["H_blocks"], full["edge_pairs"])


def test_lidar_solve_parity(pk):
    prob = scenes.lidar_street_problem(seed=1471, n_frames=3, n_points=5000)
    iters = 12
    ref = O.lm_solve(prob, params=dict(max_iters=iters))
    g = pk.Problem.from_scene(prob, max_iters=iters)
    try:
        T, info = g.solve(prob["poses0"])
    finally:
        g.close()
    assert info["iters"] == ref["iters"]
    dr = max(O.pose_error(a, b)[0] for a, b in zip(T, ref["poses"]))
    dt = max(O.pose_error(a, b)[1] for a, b in zip(T, ref["poses"]))
    assert dr <= POSE_TOL and dt <= POSE_TOL, (dr, dt, info, ref["status"], ref["iters"])
    # the solve moved the poses well beyond the tolerance
    moved = max(O.pose_error(a, b)[1] for a, b in zip(ref["poses"], prob["poses0"]))
    assert moved > 100 * POSE_TOL
    assert abs(info["final_loss"] + ref["F"]) <= LOSS_TOL * abs(ref["F"])

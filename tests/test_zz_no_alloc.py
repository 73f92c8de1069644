"""The allocation-free evaluation (rkhsba_eval_static) against rkhsba_eval.

rkhsba_eval_static serves callers that cannot allocate device memory; it runs
the same kernels in a fixed scratch array inside the library.  It must give
the results of the context path within the parity tolerances, on two calls in
a row (the second reuses the array the first left behind), and refuse
problems larger than its stated limits.  This file is collected last.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

LOSS_TOL, GRAD_TOL, H_TOL = 1e-5, 1e-4, 1e-4


def _reln(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01254_gb300 as pk
    from paper_2403_01254_gb300 import rkhsba as rb
    pk.load()
    return torch, pk, rb


def _device_inputs(torch, prob):
    xyz = torch.from_numpy(np.ascontiguousarray(np.concatenate(prob["xyz"]))).cuda()
    sem = None
    if prob.get("sem") is not None:
        sem = torch.from_numpy(np.ascontiguousarray(np.concatenate(prob["sem"]).astype(np.float32))).cuda()
    return xyz, sem


@pytest.mark.parametrize("seed", [51, 52])
def test_static_eval_matches_context_eval_twice(env, seed):
    torch, pk, rb = env
    probs = [scenes.tiny_problem(seed=seed, n_frames=3, n=400, extent=1.2, ell=0.12),
             scenes.lidar_street_problem(seed=seed, n_frames=3, n_points=3000)]
    for prob in probs:
        T = prob["poses0"]
        g = pk.Problem.from_scene(prob)
        try:
            ref = g.eval(T)
        finally:
            g.close()
        xyz, sem = _device_inputs(torch, prob)
        P = prob["params"]
        params = pk.make_params(P["ell"], P.get("cutoff_mult", 3.0), P.get("sigma", 1.0), 0.0,
                                prob["sem"][0].shape[1], P.get("sem_bf16", 0))
        n = [len(x) for x in prob["xyz"]]
        torch.cuda.synchronize()
        for _ in range(2):
            out = rb.rkhsba_eval_static(n, xyz.data_ptr(), sem.data_ptr(), None, prob["edges"], params, T)
            assert abs(out["loss"] - ref["loss"]) <= LOSS_TOL * abs(ref["loss"])
            assert _reln(out["grad"], ref["grad"]) <= GRAD_TOL
            assert _reln(out["H"], ref["H"]) <= H_TOL


def test_static_eval_refuses_problems_beyond_its_limits(env):
    torch, pk, rb = env
    prob = scenes.tiny_problem(seed=53, n_frames=2, n=20000, extent=2.0, ell=0.1)
    xyz, sem = _device_inputs(torch, prob)
    params = pk.make_params(0.1, 3.0, 1.0, 0.0, prob["sem"][0].shape[1], 0)
    with pytest.raises(pk.RkhsbaError) as ei:
        rb.rkhsba_eval_static([20000, 20000], xyz.data_ptr(), sem.data_ptr(), None, prob["edges"],
                              params, prob["poses0"])
    assert ei.value.status == 1 and "32768" in str(ei.value)

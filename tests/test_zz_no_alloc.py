"""The allocation-free evaluation (rkhsba_eval_static) against rkhsba_eval and
the FP64 oracle.

rkhsba_eval_static serves callers that cannot allocate device memory (code
inside another runtime that owns the device memory, real-time loops that must
not allocate); it runs the same kernels in a fixed scratch array inside the
library.  It must give the results of the context path and of the oracle
within the parity tolerances, on two calls in a row (the second reuses the
array the first left behind), for every label layout the kernels branch on
(FP32 and BF16 labels, colours, no labels, the top-k variant), and refuse
problems larger than its stated limits.  This file is collected last.
"""
import numpy as np
import pytest

import oracle as O
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


def _device_inputs(torch, prob, color):
    xyz = torch.from_numpy(np.ascontiguousarray(np.concatenate(prob["xyz"]))).cuda()
    sem = rgb = None
    if prob.get("sem") is not None:
        sem = torch.from_numpy(np.ascontiguousarray(np.concatenate(prob["sem"]).astype(np.float32))).cuda()
    if color:
        rgb = torch.from_numpy(np.ascontiguousarray(np.concatenate(prob["rgb"]).astype(np.float32))).cuda()
    return xyz, sem, rgb


def _variant(name, seed):
    if name == "lidar_fp32":
        return scenes.lidar_street_problem(seed=seed, n_frames=3, n_points=3000)
    prob = scenes.tiny_problem(seed=seed, n_frames=3, n=400, extent=1.2, ell=0.12, color=(name == "color"))
    if name == "bf16":
        prob["sem"] = [scenes.round_to_bf16(s) for s in prob["sem"]]
        prob["params"] = dict(prob["params"], sem_bf16=1)
    elif name == "no_labels":
        prob["sem"] = None
    elif name == "top_k":
        prob["params"] = dict(prob["params"], top_k=4)
    return prob


@pytest.mark.parametrize("name", ["fp32", "bf16", "color", "no_labels", "top_k", "lidar_fp32"])
def test_static_eval_matches_context_eval_and_oracle_twice(env, name):
    torch, pk, rb = env
    prob = _variant(name, 51)
    T = prob["poses0"]
    ref = O.evaluate(prob, T)
    g = pk.Problem.from_scene(prob)
    try:
        ctx = g.eval(T)
    finally:
        g.close()
    P = prob["params"]
    color = prob.get("rgb") is not None and P.get("ell_color", 0.0) > 0
    xyz, sem, rgb = _device_inputs(torch, prob, color)
    sem_dim = 0 if prob.get("sem") is None else prob["sem"][0].shape[1]
    params = pk.make_params(P["ell"], P.get("cutoff_mult", 3.0), P.get("sigma", 1.0), P.get("ell_color", 0.0),
                            sem_dim, P.get("sem_bf16", 0), top_k=P.get("top_k", 0))
    n = [len(x) for x in prob["xyz"]]
    torch.cuda.synchronize()
    for _ in range(2):
        out = rb.rkhsba_eval_static(n, xyz.data_ptr(), None if sem is None else sem.data_ptr(),
                                    None if rgb is None else rgb.data_ptr(), prob["edges"], params, T)
        for want in (ctx, ref):
            assert abs(out["loss"] - want["loss"]) <= LOSS_TOL * abs(want["loss"])
            assert _reln(out["grad"], want["grad"]) <= GRAD_TOL
            assert _reln(out["H"], want["H"]) <= H_TOL


def test_static_eval_refuses_problems_beyond_its_limits(env):
    torch, pk, rb = env
    prob = scenes.tiny_problem(seed=53, n_frames=2, n=20000, extent=2.0, ell=0.1)
    xyz, sem, _ = _device_inputs(torch, prob, False)
    params = pk.make_params(0.1, 3.0, 1.0, 0.0, prob["sem"][0].shape[1], 0)
    with pytest.raises(pk.RkhsbaError) as ei:
        rb.rkhsba_eval_static([20000, 20000], xyz.data_ptr(), sem.data_ptr(), None, prob["edges"],
                              params, prob["poses0"])
    assert ei.value.status == 1 and "32768" in str(ei.value)

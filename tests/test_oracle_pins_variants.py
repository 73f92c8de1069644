"""Pins of the oracle's sparse-sum variants (Sec. VI time analysis: only the
8 neighbours of largest kernel value; Sec. VII: pairs with a small semantic
kernel skipped): a pure-Python selection on small inputs, the reduction to
the full sum when nothing is cut, and finite differences of the variant's
loss."""
import math

import numpy as np
import pytest

import oracle as O
import scenes


def _tiny(seed=61, n=90):
    p = scenes.tiny_problem(seed=seed, n_frames=3, n=n, extent=0.6, ell=0.12)
    return p


def _python_F(prob, poses, top_k, sem_min):
    """F by explicit loops: per edge, per point j of the second frame, the
    candidates i inside r_c with <l_i,l_j> >= sem_min, sorted by w (desc) then i."""
    P = dict(O.DEFAULTS)
    P.update(prob["params"])
    rc2 = (P["cutoff_mult"] * P["ell"]) ** 2
    F = 0.0
    for a, b in prob["edges"]:
        xa = prob["xyz"][a] @ poses[a][:3, :3].T + poses[a][:3, 3]
        xb = prob["xyz"][b] @ poses[b][:3, :3].T + poses[b][:3, 3]
        la, lb = prob["sem"][a].astype(np.float64), prob["sem"][b].astype(np.float64)
        for j in range(len(xb)):
            cand = []
            for i in range(len(xa)):
                d2 = float(((xa[i] - xb[j]) ** 2).sum())
                if d2 >= rc2:
                    continue
                s = float(la[i] @ lb[j])
                if sem_min > 0 and s < sem_min:
                    continue
                cand.append((-s * math.exp(-d2 / (2 * P["ell"] ** 2)), i))
            cand.sort()
            if top_k > 0:
                cand = cand[:top_k]
            F -= sum(c[0] for c in cand)
    return F


@pytest.mark.parametrize("top_k,sem_min", [(0, 0.3), (1, 0.0), (3, 0.0), (2, 0.2)])
def test_variants_equal_python_selection(top_k, sem_min):
    prob = _tiny()
    prob["params"] = dict(prob["params"], top_k=top_k, sem_min=sem_min)
    ref = O.evaluate(prob, prob["poses0"])
    np.testing.assert_allclose(ref["F"], _python_F(prob, prob["poses0"], top_k, sem_min), rtol=1e-12)
    full = O.evaluate(dict(prob, params=dict(prob["params"], top_k=0, sem_min=0.0)), prob["poses0"])
    assert ref["n_pairs"] < full["n_pairs"]


def test_large_top_k_is_the_full_sum():
    prob = _tiny()
    full = O.evaluate(prob, prob["poses0"])
    big = O.evaluate(dict(prob, params=dict(prob["params"], top_k=10 ** 6)), prob["poses0"])
    assert big["n_pairs"] == full["n_pairs"]
    np.testing.assert_allclose(big["F"], full["F"], rtol=1e-15)
    np.testing.assert_allclose(big["H"], full["H"], rtol=1e-13, atol=1e-13)


def test_top_k_gradient_matches_finite_differences():
    prob = _tiny(seed=62, n=40)
    prob["params"] = dict(prob["params"], top_k=3, cutoff_mult=math.inf)
    T = prob["poses0"]
    g = O.evaluate(prob, T)["grad"]
    h = 1e-6
    fd = np.zeros_like(g)
    for m in range(1, 3):
        for k in range(6):
            xi = np.zeros(6)
            xi[k] = h
            Tp, Tm = T.copy(), T.copy()
            Tp[m] = T[m] @ O.se3_exp(xi)
            Tm[m] = T[m] @ O.se3_exp(-xi)
            fd[6 * m + k] = (O.evaluate(prob, Tp)["loss"] - O.evaluate(prob, Tm)["loss"]) / (2 * h)
    np.testing.assert_allclose(g[6:], fd[6:], rtol=1e-5, atol=1e-7)

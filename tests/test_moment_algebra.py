"""The per-edge assembly of the CUDA path works from 28 weighted moments of
the pairs instead of per-pair Jacobians (a4/a5 of the hot path).  This CPU
test restates that algebra in FP64 and checks it against the oracle's direct
per-pair sums b = sum w J^T d and H = sum w J^T J (Sec. V-A, Eq. irls_final)
to 1e-12: it pins the formulas independently of the kernel's FP32 and
fixed-point arithmetic.

Moments, in frame-a coordinates, with x the frame-a point, y' = T_ab y the
transformed frame-b point and d = x - y':
  W = sum w, D = sum w d, Sy = sum w y', Myy = sum w y'y'^T,
  Mdy = sum w d y'^T, Q = sum w d d^T.
"""
import numpy as np
import pytest

import oracle as O


def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def assemble_from_moments(W, D, Sy, Myy, Mdy, Q, R, t):
    """b (12) and H (12 x 12) of one edge, [rho_a, phi_a, rho_b, phi_b], from
    the moments and the relative pose T_ab = [R | t]."""
    Sx = Sy + D                                          # sum w x
    St = Sy - W * t                                      # sum w (y' - t)
    Mxx = Myy + Mdy + Mdy.T + Q                          # sum w x x^T
    Mxt = Myy + Mdy - np.outer(Sx, t)                    # sum w x (y' - t)^T
    Mtt = Myy - np.outer(Sy, t) - np.outer(t, Sy) + W * np.outer(t, t)
    Gx = np.array([Mdy[2, 1] - Mdy[1, 2], Mdy[0, 2] - Mdy[2, 0], Mdy[1, 0] - Mdy[0, 1]])   # sum w x (x) d
    Gt = Gx - np.cross(t, D)                             # sum w (y' - t) (x) d
    b = np.concatenate([D, Gx, -R.T @ D, -R.T @ Gt])
    Sb = R.T @ St
    Mb = R.T @ Mtt @ R
    I3 = np.eye(3)
    H = np.zeros((12, 12))
    H[:3, :3] = W * I3
    H[:3, 3:6] = -_skew(Sx)
    H[3:6, :3] = _skew(Sx)
    H[3:6, 3:6] = np.trace(Mxx) * I3 - Mxx
    H[6:9, 6:9] = W * I3
    H[6:9, 9:] = -_skew(Sb)
    H[9:, 6:9] = _skew(Sb)
    H[9:, 9:] = np.trace(Mb) * I3 - Mb
    Hab = np.block([[-W * R, _skew(St) @ R], [-_skew(Sx) @ R, (Mxt.T - np.trace(Mxt) * I3) @ R]])
    H[:6, 6:] = Hab
    H[6:, :6] = Hab.T
    return b, H


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_moment_assembly_equals_per_pair_sums(seed):
    rng = np.random.default_rng(seed)
    n = 60
    xa = rng.uniform(-1, 1, (n, 3)) * 3.0 + 20.0          # away from the origin: the moments carry it
    xb = xa + rng.normal(scale=0.05, size=xa.shape)
    sa = rng.dirichlet(np.ones(4), n).astype(np.float32)
    sb = rng.dirichlet(np.ones(4), n).astype(np.float32)
    Ta = O.se3_exp(np.concatenate([rng.normal(size=3), rng.normal(size=3) * 0.7]))
    Tb = Ta @ O.se3_exp(np.concatenate([rng.normal(size=3) * 0.05, rng.normal(size=3) * 0.05]))
    P = dict(O.DEFAULTS, ell=0.4, cutoff_mult=np.inf)
    ref = O.edge_terms(xa, xb, Ta, Tb, sa, sb, params=P)

    Tab = np.linalg.inv(Ta) @ Tb
    R, t = Tab[:3, :3], Tab[:3, 3]
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    x = xa[i]
    y = xb[j] @ R.T + t
    d = x - y
    w = np.einsum("nk,nk->n", sa[i].astype(np.float64), sb[j]) * np.exp(-np.einsum("nk,nk->n", d, d) / (2 * 0.4 ** 2))
    W = w.sum()
    D = (w[:, None] * d).sum(0)
    Sy = (w[:, None] * y).sum(0)
    Myy = np.einsum("n,nk,nl->kl", w, y, y)
    Mdy = np.einsum("n,nk,nl->kl", w, d, y)
    Q = np.einsum("n,nk,nl->kl", w, d, d)
    b, H = assemble_from_moments(W, D, Sy, Myy, Mdy, Q, R, t)

    np.testing.assert_allclose(W, ref["W"], rtol=1e-12)
    np.testing.assert_allclose(b, ref["b"], rtol=1e-12, atol=1e-12 * np.abs(ref["b"]).max())
    np.testing.assert_allclose(H, ref["H"], rtol=1e-12, atol=1e-12 * np.abs(ref["H"]).max())

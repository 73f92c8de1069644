"""The dense tile unit of the pair kernel forms the 28 edge moments from
per-query sums over candidates (k_q = sum_c w, X1_q = sum_c w x_c, X2_q =
sum_c w x_c x_c^T) instead of per-pair sums of d = x - y', and carries the
weights and the candidate features through the tensor cores as FP16 hi + lo
pairs.  This CPU test restates both pieces in numpy and pins them apart from
the kernel:

  * the unit-end formulas W = sum k, D = sum (X1 - k y), Sy = sum k y,
    Myy = sum k y y^T, Mdy = sum (X1 - k y) y^T, Q = sum (X2 - X1 y^T -
    y X1^T + k y y^T) equal the per-pair definitions (Sec. V-A, the moments
    behind Eq. irls_final) to 1e-12 in FP64;
  * the split a = a_hi + a_lo (each rounded to FP16) with the product
    a_hi b_hi + a_hi b_lo + a_lo b_hi keeps the relative error of w x below
    2^-20 over the scaled operand ranges the kernel uses (w 2^KW <= 2^14,
    |x 2^-EX| <= 2.6) wherever the lo parts are normal FP16 numbers; below
    that (scaled weights under 2^-3) the error stays under half an FP16
    subnormal step, 2^-25 in scaled units (2^-38 of a weight for KW = 13);
    and the errors do not add up to a bias in long sums.
"""
import numpy as np


def _split(a):
    hi = a.astype(np.float16).astype(np.float64)
    lo = (a - hi).astype(np.float16).astype(np.float64)
    return hi, lo


def test_per_query_sums_give_the_pair_moments():
    rng = np.random.default_rng(5)
    nq, nc = 23, 57
    y = rng.uniform(-1.3, 1.3, (nq, 3))                 # queries, home-cell coordinates
    x = rng.uniform(-1.3, 1.3, (nc, 3))                 # candidates
    w = rng.uniform(0.0, 1.0, (nc, nq)) * (rng.uniform(size=(nc, nq)) < 0.6)
    d = x[:, None, :] - y[None, :, :]                   # [c, q, 3]
    ref = dict(W=w.sum(), D=np.einsum("cq,cqm->m", w, d), Sy=np.einsum("cq,qm->m", w, y),
               Myy=np.einsum("cq,qm,ql->ml", w, y, y), Mdy=np.einsum("cq,cqm,ql->ml", w, d, y),
               Q=np.einsum("cq,cqm,cql->ml", w, d, d))
    k = w.sum(0)                                        # per query
    X1 = w.T @ x                                        # [q, 3]
    X2 = np.einsum("cq,cm,cl->qml", w, x, x)            # [q, 3, 3]
    D = X1 - k[:, None] * y
    got = dict(W=k.sum(), D=D.sum(0), Sy=(k[:, None] * y).sum(0),
               Myy=np.einsum("q,qm,ql->ml", k, y, y), Mdy=np.einsum("qm,ql->ml", D, y),
               Q=(X2 - np.einsum("qm,ql->qml", X1, y) - np.einsum("qm,ql->qml", y, X1)
                  + np.einsum("q,qm,ql->qml", k, y, y)).sum(0))
    for key in ref:
        scale = max(np.abs(ref[key]).max(), 1.0)
        assert np.abs(got[key] - ref[key]).max() <= 1e-12 * scale, key


def test_fp16_split_products_keep_22_bits():
    rng = np.random.default_rng(6)
    n = 200000
    w = np.exp(rng.uniform(np.log(1e-3), np.log(2.0 ** 14), n))      # scaled weights
    f = rng.uniform(-2.6, 2.6, n)                                    # scaled features
    f[::97] = 1.0                                                    # the constant feature
    wh, wl = _split(w)
    fh, fl = _split(f)
    prod = wh * fh + wh * fl + wl * fh
    exact = w * f
    err = np.abs(prod - exact)
    normal = (w >= 2.0 ** -3) & (np.abs(f) >= 2.0 ** -3)   # lo parts in FP16's normal range
    assert (err[normal] / np.abs(exact[normal])).max() < 2.0 ** -20
    # elsewhere an absolute bound: half a subnormal step of each lo part
    assert (err <= 2.0 ** -20 * np.abs(exact) + 2.0 ** -25 * (np.abs(f) + w)).all()
    # long sums: the rounding errors are not one-signed (no bias)
    s_err = (prod - exact).sum() / np.abs(exact).sum()
    assert abs(s_err) < 1e-8
    # the weights alone (the loss column) round-trip to 22 bits, or to half a
    # subnormal step
    assert (np.abs(wh + wl - w) <= np.maximum(2.0 ** -21 * w, 2.0 ** -25)).all()

"""The oracle's sums split over slices of each edge's second frame (the form
the full-size GPU checks and the all-core CPU baseline use) equal the plain
oracle: every sum of Eq. (inner_product_actual_ba) runs over the points of
frame b, and the top-k and semantic-pruning selections are per point of
frame b, so slicing frame b changes only the FP64 summation order."""
import numpy as np
import pytest

import oracle as O
import scenes
from oracle.split_sum import evaluate_split


@pytest.mark.parametrize("over", [{}, {"top_k": 3}, {"sem_min": 0.2}])
@pytest.mark.parametrize("workers", [1, 2])
def test_split_sum_equals_plain_oracle(over, workers):
    prob = scenes.tiny_problem(seed=91, n_frames=3, n=500, extent=1.0, ell=0.15, color=True)
    prob["params"] = dict(prob["params"], **over)
    T = prob["poses0"]
    ref = O.evaluate(prob, T)
    ids = list(range(len(prob["edges"])))
    got = evaluate_split(prob, T, ids, slice_points=97, workers=workers)
    assert np.array_equal(got["edge_pairs"], ref["edge_pairs"])
    assert abs(got["loss"] - ref["loss"]) <= 1e-12 * abs(ref["loss"])
    assert np.abs(got["grad"] - ref["grad"]).max() <= 1e-12 * np.abs(ref["grad"]).max()
    assert np.abs(got["H"] - ref["H"]).max() <= 1e-12 * np.abs(ref["H"]).max()
    for e in ids:
        assert np.abs(got["H_blocks"][e] - ref["H_blocks"][e]).max() <= 1e-12 * np.abs(ref["H_blocks"][e]).max()


def test_split_sum_on_an_edge_subset():
    prob = scenes.lidar_street_problem(seed=92, n_frames=4, n_points=1500)
    T = prob["poses0"]
    ids = [1, 4]
    sub = dict(prob, edges=np.asarray(prob["edges"])[ids])
    ref = O.evaluate(sub, T)
    got = evaluate_split(prob, T, ids, slice_points=400, workers=2)
    assert np.array_equal(got["edge_pairs"], ref["edge_pairs"])
    assert abs(got["loss"] - ref["loss"]) <= 1e-12 * abs(ref["loss"])
    assert np.abs(got["grad"] - ref["grad"]).max() <= 1e-12 * np.abs(ref["grad"]).max()

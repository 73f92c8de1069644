"""Failure detection on the device: a bounded wait that runs out.

The radix sort behind the grid build and the query binning hands tile counts
from block to block by decoupled look-back; every wait on another block's
record polls a bounded number of times, then raises an error word that the
entry points report as RKHSBA_ETIMEOUT.  The self-test entry point makes one
such wait run out on purpose (a record that nothing publishes): the status is
ETIMEOUT, no write leaves the output arrays, and the GPU context stays usable
for the next evaluation, whose results are unchanged.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01254_gb300 as pk
    pk.load()
    return pk


def test_lookback_wait_runs_out_and_reports_etimeout(pk):
    from paper_2403_01254_gb300 import rkhsba as rb
    prob = scenes.lidar_street_problem(seed=61, n_frames=3, n_points=3000)
    g = pk.Problem.from_scene(prob)
    try:
        before = g.eval(prob["poses0"])
        for limit in (1, 1000):
            status, in_bounds = rb.rkhsba_selftest_lookback_timeout(limit)
            assert status == "ETIMEOUT"
            assert in_bounds
        after = g.eval(prob["poses0"])
    finally:
        g.close()
    assert after["loss"] == before["loss"]
    assert np.array_equal(after["grad"], before["grad"])
    assert np.array_equal(after["H"], before["H"])


def test_selftest_rejects_bad_limits(pk):
    from paper_2403_01254_gb300 import rkhsba as rb
    for bad in (0, -5, (1 << 20) + 1):
        with pytest.raises(pk.RkhsbaError) as ei:
            rb.rkhsba_selftest_lookback_timeout(bad)
        assert ei.value.status == 1

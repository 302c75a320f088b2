"""Host logic of the serving loop that needs no GPU: the launch policy of a request,
its launch batches and HBM footprint (what admission compares with the memory
budget), and the seeded serving mix."""
import numpy as np
import pytest

from paper_2210_15874_gb300 import serving as S
from paper_2210_15874_gb300 import workloads as W


def req(n, K, p=2, damping=5e-3):
    g, b = W.angles(p, 7)
    return S.Request(n, W.regular_graph(n, 3 if n % 2 == 0 else 4, 11), g, b, K, 99, damping=damping)


def test_launch_policy():
    small_one, small_many, large = req(10, 512), req(12, 10**6), req(14, 512)
    assert small_many.chunks() > 1 and small_one.chunks() == 1
    assert S.launch_mode_for(small_one) == 1  # device-driven
    assert S.launch_mode_for(small_many) == 2  # captured once, replayed per launch batch
    assert S.launch_mode_for(large) == 0  # sized on the host
    for r in (small_one, small_many, large):
        assert [S.launch_mode_for(r, pol) for pol in ("host", "device", "graph")] == [0, 1, 2]
    with pytest.raises(ValueError):
        S.launch_mode_for(small_one, "fastest")


def test_launch_batches_and_footprint():
    r = req(24, 8192, p=6)
    assert r.launch_batch() == S.STATE_BUDGET_BYTES // (8 << 24) == 64
    assert r.chunks() == 128
    assert req(10, 300).launch_batch() == 300 and req(10, 300).chunks() == 1
    # the footprint holds the launch batch of statevectors, grows with n and with the depth
    for n in (10, 16, 20, 24):
        f = req(n, 4096).footprint()
        assert f >= req(n, 4096).launch_batch() * (8 << n)
        assert req(n, 4096, p=6).footprint() > req(n, 4096, p=1).footprint()
    assert req(20, 4096).footprint() > req(16, 4096).footprint()
    assert req(24, 8192).footprint() < S.STATE_BUDGET_BYTES + (1 << 30)


def test_serving_mix_is_seeded_and_in_range():
    a, b = S.serving_mix(40), S.serving_mix(40)
    assert len(a) == 40
    for x, y in zip(a, b):
        assert (x.n, x.trajectories, x.seed) == (y.n, y.trajectories, y.seed)
        np.testing.assert_array_equal(x.edges, y.edges)
        np.testing.assert_array_equal(x.gammas, y.gammas)
    assert [r.n for r in S.serving_mix(40, seed=1)] != [r.n for r in a]
    for r in a:
        assert 10 <= r.n <= 24 and 1 <= len(r.gammas) <= 6 and len(r.betas) == len(r.gammas)
        assert 256 <= r.trajectories < 8192
        assert r.damping == 5e-3 and r.p1 == 1e-3 and r.p2 == 1e-2
        deg = np.bincount(r.edges.reshape(-1), minlength=r.n)
        assert np.all(deg == (3 if r.n % 2 == 0 else 4))
        assert len({tuple(sorted(e)) for e in r.edges.tolist()}) == len(r.edges)


def test_percentile():
    assert S.percentile([1.0, 2.0, 3.0, 4.0], 50) == 2.5
    assert S.percentile(list(range(101)), 99) == 99.0
    assert np.isnan(S.percentile([], 50))

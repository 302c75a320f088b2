"""Continuous batching (paper_2210_15874_gb300.serving): requests of mixed n,
depth, trajectory count and noise are admitted by HBM footprint as slots free
up and run concurrently on separate streams, with device-driven launches (and
CUDA graphs replayed over the chunks of a request that runs in several).  Each
result must equal the same request run alone with host-sized launches."""
import numpy as np
import pytest

from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import serving
    return serving


def make_requests(serving, count, rng):
    reqs = []
    for i in range(count):
        n = int(rng.integers(8, 15))
        p = int(rng.integers(1, 4))
        K = int(np.exp(rng.uniform(np.log(32), np.log(512))))
        g, b = W.angles(p, 700 + i)
        damp = 5e-3 if i % 2 == 0 else 0.0
        d = 3 if n % 2 == 0 else 4  # 3-regular graphs need an even vertex count
        reqs.append(serving.Request(n, W.regular_graph(n, d, 800 + n), g, b, K, 0x5E7 + i, damping=damp,
                                    want_probs=True))
    return reqs


def test_results_equal_alone_and_in_the_mix(mods):
    serving = mods
    reqs = make_requests(serving, 12, np.random.default_rng(5))
    alone = [serving.run_alone(r) for r in reqs]
    srv = serving.Server(max_inflight=4)
    futs = [srv.submit(r) for r in reqs]
    mixed = [f.result(timeout=300) for f in futs]
    srv.close()
    for a, m in zip(alone, mixed):
        assert abs(a.mean - m.mean) < 1e-12 and abs(a.std_err - m.std_err) < 1e-12
        np.testing.assert_allclose(m.probs, a.probs, rtol=1e-12, atol=1e-15)
    # the requests overlapped: some started before others finished, on the host and on the
    # device (CUDA events on each request's stream, against the server's reference event)
    spans = sorted((m.started, m.finished) for m in mixed)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    dev = sorted((m.device_start, m.device_end) for m in mixed)
    assert all(a <= b for a, b in dev)
    assert any(dev[i + 1][0] < dev[i][1] for i in range(len(dev) - 1))


def test_admission_by_footprint(mods):
    """Admission never lets the footprints in flight exceed the budget: with the
    largest request's footprint as the budget, that request runs alone; a budget
    that holds the two smallest together keeps at most two in flight; a request
    above the budget is refused at submission."""
    serving = mods
    reqs = make_requests(serving, 5, np.random.default_rng(6))
    fp = sorted(r.footprint() for r in reqs)
    budget = fp[-1]
    srv = serving.Server(max_inflight=4, mem_budget=budget)
    futs = [srv.submit(r) for r in reqs]
    res = [f.result(timeout=300) for f in futs]
    srv.close()
    assert len(res) == 5 and all(np.isfinite(r.mean) for r in res)
    assert len(srv.admissions) == 5
    assert all(used <= budget for _, _, used in srv.admissions)
    big = max(range(5), key=lambda i: reqs[i].footprint())
    for i in range(5):  # nothing else fits beside the largest request
        if i != big:
            assert res[i].finished <= res[big].started or res[i].started >= res[big].finished
    # room for the two smallest together (and not for three)
    budget2 = fp[0] + fp[1]
    small = [r for r in reqs if r.footprint() <= budget2]
    srv = serving.Server(max_inflight=4, mem_budget=budget2)
    res2 = [f.result(timeout=300) for f in [srv.submit(r) for r in small]]
    srv.close()
    assert len(res2) == len(small)
    assert all(used <= budget2 and inflight <= 2 for _, inflight, used in srv.admissions)
    with pytest.raises(ValueError):
        srv2 = serving.Server(max_inflight=1, mem_budget=1024)
        try:
            srv2.submit(reqs[0])
        finally:
            srv2.close()


def test_chunked_requests_replay_their_graphs(mods, monkeypatch):
    """With launch batches smaller than the requests, the graph launch policy captures each
    damping request's first chunk in a CUDA graph and replays it for the others; the
    results equal host-sized runs of the same requests, alone."""
    serving = mods
    monkeypatch.setattr(serving, "STATE_BUDGET_BYTES", 2 << 20)  # small launch batches: several chunks
    reqs = [r for r in make_requests(serving, 16, np.random.default_rng(8)) if r.damping > 0 and r.chunks() >= 2]
    assert len(reqs) >= 3
    alone = [serving.run_alone(r, "host") for r in reqs]
    srv = serving.Server(max_inflight=3, launch_policy="graph")
    mixed = [f.result(timeout=300) for f in [srv.submit(r) for r in reqs]]
    srv.close()
    for r, a, m in zip(reqs, alone, mixed):
        assert m.launch["mode"] == 2
        assert m.launch["captures"] + m.launch["replays"] == r.chunks()
        assert m.launch["replays"] >= r.chunks() - 2  # only a shorter last chunk captures again
        assert a.mean == m.mean and a.std_err == m.std_err
        np.testing.assert_array_equal(m.probs, a.probs)

"""qn_run_qaoa_noalloc: the allocation-free batch entry point.

It serves callers that may not allocate device memory (memory owned by another
runtime or pool, a fixed budget, or loops that cannot afford cudaMalloc's
synchronisation): they pass the statevector workspace and output buffers, and
the library's own scratch lives in a static device array that every call
shares.  These tests call it through the C ABI and check its results against
the handle path (qn_run_qaoa) and against the FP64 oracle, with an unrelated
call in between the compared ones so that the shared array holds another
batch's tables, counters and status word when the second compared call starts.
The file is named so pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tolerances import TOL_CT
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn
    return qn, torch


def _args(qn, w):
    e = np.ascontiguousarray(np.asarray(w.edges, dtype=np.int32).reshape(-1))
    g = np.ascontiguousarray(w.gammas, dtype=np.float64)
    b = np.ascontiguousarray(w.betas, dtype=np.float64)
    graph = qn.qn_graph(w.n, len(e) // 2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    nk = w.noise_kwargs()
    noise = qn.qn_noise(nk["p1"], nk["p2"], nk["damping"], nk["twoq_mode"], nk["param"])
    return e, g, b, graph, noise


def raw_call(qn, w, first, count, psi, c_out, probs, stream):
    """One qn_run_qaoa_noalloc call; returns its status (keeps the host arrays alive)."""
    e, g, b, graph, noise = _args(qn, w)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return qn.qn_run_qaoa_noalloc(w.n, ctypes.byref(graph), len(g), dp(g), dp(b), ctypes.byref(noise),
                                  ctypes.c_uint64(w.seed), first, count, psi, c_out, probs,
                                  ctypes.c_void_p(stream.cuda_stream) if stream is not None else None)


def call_noalloc(qn, torch, w, first, count, stream):
    psi = torch.empty((count, 1 << w.n, 2), dtype=torch.float32, device="cuda")
    c_out = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
    probs = torch.full((1 << w.n,), float("nan"), dtype=torch.float64, device="cuda")
    st = raw_call(qn, w, first, count, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(c_out.data_ptr()),
                  ctypes.c_void_p(probs.data_ptr()), stream)
    qn.check(st, "qn_run_qaoa_noalloc")
    torch.cuda.synchronize()
    return c_out.cpu().numpy(), probs.cpu().numpy()


def test_noalloc_matches_handle_path_and_oracle_with_other_calls_between(env):
    qn, torch = env
    w = W.qaoa_workload("noalloc_n14", 14, 2, index=9, trajectories=12, batch=12, p1=5e-3, p2=2e-2,
                        damping=0.05)
    # an unrelated batch: other n, count, depth, seed and noise, so the shared scratch
    # holds other tables, counters and status when the next compared call starts
    other = W.qaoa_workload("noalloc_other", 11, 3, index=19, trajectories=300, batch=300, p1=2e-2, p2=5e-2,
                            damping=0.2, d=4)
    first, count = 5, 12
    with qn.Batch(w.n, count, w.seed) as h:
        h.set_offset(first)
        h.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        ref_probs = h.probs() * count
        ref_c = h.traj_debug(0, count, amps=False, branches=False)["c_traj"]
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    orc = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, first, count,
                          want_amps=False)
    tol_c = TOL_CT
    stream = torch.cuda.Stream()
    runs = []
    for _ in range(2):
        runs.append(call_noalloc(qn, torch, w, first, count, stream))
        call_noalloc(qn, torch, other, 0, other.trajectories, stream)
    for c_out, probs in runs:
        assert np.all(np.isfinite(c_out)) and np.all(np.isfinite(probs))
        # against the handle path
        assert np.abs(c_out - ref_c).max() < tol_c
        np.testing.assert_allclose(probs / count, ref_probs / count, atol=2e-6)
        assert abs(probs.sum() / count - 1) < 1e-6
        # against the FP64 oracle on the same trajectories (same Philox draws)
        assert np.abs(c_out - orc["c_traj"]).max() < tol_c
        np.testing.assert_allclose(probs, orc["probs_sum"], rtol=1e-5, atol=1e-9)
        assert oracle.error(probs / count, orc["probs_sum"] / count) < 1e-9
    # the two compared calls agree bit for bit
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])


def test_noalloc_at_the_scratch_limit(env):
    """The largest batch that fits the 8 MiB scratch (found by probing: a call that
    does not fit returns QN_EINVAL before anything is queued) runs and matches the
    handle path; one trajectory more is refused."""
    qn, torch = env
    w = W.qaoa_workload("noalloc_limit", 10, 1, index=21, trajectories=1, batch=1, p1=5e-3, p2=2e-2,
                        damping=0.02)
    stream = torch.cuda.Stream()
    dim = 1 << w.n
    cap = 65535
    psi = torch.empty((cap, dim, 2), dtype=torch.float32, device="cuda")  # 537 MB at n=10
    c_out = torch.empty((cap,), dtype=torch.float64, device="cuda")
    probs = torch.empty((dim,), dtype=torch.float64, device="cuda")
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in (psi, c_out, probs)]

    def fits(count):
        st = raw_call(qn, w, 0, count, *ptrs, stream)
        torch.cuda.synchronize()
        if st == qn.QN_EINVAL:
            assert b"scratch" in qn.qn_last_error()
            return False
        qn.check(st, "qn_run_qaoa_noalloc")
        return True

    assert fits(1) and not fits(cap)
    lo, hi = 1, cap  # fits(lo), not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    assert lo > 1000  # the scratch holds thousands of 10-qubit trajectories
    assert fits(lo) and not fits(lo + 1)
    c = c_out[:lo].cpu().numpy()
    pr = probs.cpu().numpy()
    with qn.Batch(w.n, lo, w.seed) as h:
        h.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        ref_probs = h.probs()
        m, _ = h.expectation()
    assert abs(c.mean() - m) < 1e-9
    np.testing.assert_allclose(pr / lo, ref_probs, atol=1e-9)


def test_noalloc_rejects_batches_beyond_scratch(env):
    qn, torch = env
    w = W.damping_n20()
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    st = raw_call(qn, w, 0, 4096, fake, fake, fake, None)
    assert st == qn.QN_EINVAL
    assert b"scratch" in qn.qn_last_error()


def test_noalloc_rejects_host_and_foreign_buffers(env):
    """A host buffer passed as psi, c_out or probs_out gives QN_EINVAL before
    anything is queued (the outputs keep their contents)."""
    qn, torch = env
    w = W.qaoa_workload("noalloc_host", 8, 1, index=3, trajectories=4, batch=4, p1=1e-3, p2=1e-2)
    count = 4
    psi = torch.empty((count, 1 << w.n, 2), dtype=torch.float32, device="cuda")
    c_out = torch.full((count,), -7.0, dtype=torch.float64, device="cuda")
    probs = torch.full((1 << w.n,), -7.0, dtype=torch.float64, device="cuda")
    host_psi = np.zeros((count, 1 << w.n, 2), dtype=np.float32)
    host_c = np.zeros(count, dtype=np.float64)
    dev = [ctypes.c_void_p(t.data_ptr()) for t in (psi, c_out, probs)]
    torch.cuda.synchronize()
    for which, host in ((0, host_psi), (1, host_c)):
        args = list(dev)
        args[which] = ctypes.c_void_p(host.ctypes.data)
        st = raw_call(qn, w, 0, count, *args, None)
        assert st == qn.QN_EINVAL
        assert b"device memory" in qn.qn_last_error()
    torch.cuda.synchronize()
    assert np.all(c_out.cpu().numpy() == -7.0) and np.all(probs.cpu().numpy() == -7.0)
    # the same buffers on the device are accepted
    qn.check(raw_call(qn, w, 0, count, *dev, None), "qn_run_qaoa_noalloc")
    torch.cuda.synchronize()
    assert abs(probs.cpu().numpy().sum() / count - 1) < 1e-6

"""qn_run_qaoa_noalloc: the allocation-free batch entry point.

It serves callers that may not allocate device memory (memory owned by another
runtime or pool, a fixed budget, or loops that cannot afford cudaMalloc's
synchronisation): they pass the statevector workspace and output buffers, and
the library's own scratch lives in a static device array.  This test calls it
through the C ABI twice in a row and compares both results with the handle
path (qn_run_qaoa) on the same trajectories.  The file is named so pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

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


def call_noalloc(qn, torch, w, first, count, stream):
    e = np.ascontiguousarray(np.asarray(w.edges, dtype=np.int32).reshape(-1))
    g = np.ascontiguousarray(w.gammas, dtype=np.float64)
    b = np.ascontiguousarray(w.betas, dtype=np.float64)
    graph = qn.qn_graph(w.n, len(e) // 2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    nk = w.noise_kwargs()
    noise = qn.qn_noise(nk["p1"], nk["p2"], nk["damping"], nk["twoq_mode"], nk["param"])
    psi = torch.empty((count, 1 << w.n, 2), dtype=torch.float32, device="cuda")
    c_out = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
    probs = torch.full((1 << w.n,), float("nan"), dtype=torch.float64, device="cuda")
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = qn.qn_run_qaoa_noalloc(w.n, ctypes.byref(graph), len(g), dp(g), dp(b), ctypes.byref(noise),
                                ctypes.c_uint64(w.seed), first, count, ctypes.c_void_p(psi.data_ptr()),
                                ctypes.c_void_p(c_out.data_ptr()), ctypes.c_void_p(probs.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
    qn.check(st, "qn_run_qaoa_noalloc")
    torch.cuda.synchronize()
    return c_out.cpu().numpy(), probs.cpu().numpy()


def test_noalloc_matches_handle_path_twice(env):
    qn, torch = env
    w = W.qaoa_workload("noalloc_n14", 14, 2, index=9, trajectories=12, batch=12, p1=5e-3, p2=2e-2,
                        damping=0.05)
    first, count = 5, 12
    with qn.Batch(w.n, count, w.seed) as h:
        h.set_offset(first)
        h.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        ref_probs = h.probs() * count
        ref_c = h.traj_debug(0, count, amps=False, branches=False)["c_traj"]
    G = w.gate_count
    tol_c = 8 * U32 * G * len(w.edges)
    stream = torch.cuda.Stream()
    runs = [call_noalloc(qn, torch, w, first, count, stream) for _ in range(2)]
    for c_out, probs in runs:
        assert np.all(np.isfinite(c_out)) and np.all(np.isfinite(probs))
        assert np.abs(c_out - ref_c).max() < tol_c
        np.testing.assert_allclose(probs / count, ref_probs / count, atol=2e-6)
        assert abs(probs.sum() / count - 1) < 1e-6


def test_noalloc_rejects_batches_beyond_scratch(env):
    qn, torch = env
    w = W.damping_n20()
    e = np.ascontiguousarray(np.asarray(w.edges, dtype=np.int32).reshape(-1))
    graph = qn.qn_graph(w.n, len(e) // 2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    g = np.ascontiguousarray(w.gammas)
    b = np.ascontiguousarray(w.betas)
    noise = qn.qn_noise(w.p1, w.p2, w.damping, 0, 0)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fake = ctypes.c_void_p(256)  # never dereferenced: the size check fails first
    st = qn.qn_run_qaoa_noalloc(w.n, ctypes.byref(graph), w.p, dp(g), dp(b), ctypes.byref(noise),
                                ctypes.c_uint64(1), 0, 4096, fake, fake, fake, None)
    assert st == qn.QN_EINVAL
    assert b"scratch" in qn.qn_last_error()

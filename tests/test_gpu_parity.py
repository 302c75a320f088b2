"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bars (each follows from the FP32 arithmetic of the path):
  * Pauli codes bit-exact (integer thresholds on the same Philox words);
  * damping branches equal except where u lies within FP32 reach of p1 (counted);
  * amplitudes within 1e-5 absolute;
  * <C>_t within TOL_CT and ensemble means within TOL_MEAN (tests/tolerances.py);
  * ensemble <C> and sigma_approx against the oracle's trajectories on the same
    seed, and <C> within 3 sigma/sqrt(K) of the density matrix.
"""
import numpy as np
import pytest

import oracle
from tolerances import TOL_CT, TOL_MEAN
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


def run_gpu(qn, w, *, launch_batch=0, count=None, t0=0):
    b = qn.Batch(w.n, w.trajectories, w.seed, launch_batch=launch_batch)
    b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
    mean, se = b.expectation()
    probs = b.probs()
    dbg = b.traj_debug(t0, count if count is not None else w.trajectories)
    info = b.run_info()
    b.close()
    return dict(mean=mean, se=se, probs=probs, info=info, **dbg)


def run_oracle(w, t0=0, count=None, want_amps=True):
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    return oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, t0,
                           count if count is not None else w.trajectories, want_amps=want_amps), gates, G, nz


def compare_trajectories(gpu, orc, w, G, allow_damp_mismatch=0):
    br_g, br_o = gpu["branches"], orc["branches"]
    assert br_g.shape == br_o.shape
    # Pauli codes: bit-exact everywhere
    np.testing.assert_array_equal(br_g & 15, br_o & 15)
    same = np.all(br_g == br_o, axis=1)
    assert (~same).sum() <= allow_damp_mismatch, f"{(~same).sum()} damping-branch mismatches"
    amp_err = np.abs(gpu["amps"][same] - orc["amps"][same]).max()
    assert amp_err < 1e-5, amp_err
    tol_c = TOL_CT
    c_err = np.abs(gpu["c_traj"][same] - orc["c_traj"][same]).max()
    assert c_err < tol_c, (c_err, tol_c)
    return amp_err, c_err


def test_plain_n8_matches_oracle(qn):
    """8-qubit p=1 QAOA, depolarizing p1=1e-3 / p2=1e-2, K=1024 in one launch."""
    w = W.plain_n8()
    gpu = run_gpu(qn, w)
    orc, gates, G, nz = run_oracle(w)
    compare_trajectories(gpu, orc, w, G)
    K = w.trajectories
    assert abs(gpu["mean"] - orc["s1"] / K) < TOL_MEAN
    np.testing.assert_allclose(gpu["probs"], orc["probs_sum"] / K, atol=1e-6)
    assert abs(gpu["probs"].sum() - 1) < 1e-6
    assert oracle.error(gpu["probs"], orc["probs_sum"] / K) < 1e-9
    dm = oracle.dm_run(w.n, w.edges, gates, G, nz)
    assert abs(gpu["mean"] - dm["c"]) < 3 * gpu["se"]
    assert gpu["info"]["gates"] == G


def test_damping_multi_tile_ragged(qn):
    """14 qubits (8 sweep tiles per trajectory), p=2, depolarizing + damping 0.05,
    K=48 in launches of 20 (20 + 20 + 8)."""
    w = W.qaoa_workload("damp_n14", 14, 2, index=7, trajectories=48, batch=20, p1=5e-3, p2=2e-2, damping=0.05)
    gpu = run_gpu(qn, w, launch_batch=20)
    orc, gates, G, nz = run_oracle(w)
    assert np.any(orc["branches"] & 0x30), "no damping jump in the sample; the case would not test jumps"
    compare_trajectories(gpu, orc, w, G, allow_damp_mismatch=1)
    K = w.trajectories
    assert abs(gpu["mean"] - orc["s1"] / K) < TOL_MEAN
    assert oracle.error(gpu["probs"], orc["probs_sum"] / K) < 1e-9


@pytest.mark.parametrize("case", [
    "n1_no_edges", "n2_one_edge", "p0_h_layer_only", "k1_single", "gamma_one", "full_depolarizing",
    "product_mode", "lambda_param", "reversed_edges", "no_noise", "n12_two_tiles"])
def test_edge_cases(qn, case):
    n, p, K, kw, edges = 5, 1, 64, dict(p1=0.05, p2=0.1, damping=0.1), None
    if case == "n1_no_edges":
        n, edges = 1, np.zeros((0, 2), dtype=np.int32)
    elif case == "n2_one_edge":
        n, edges = 2, np.array([[0, 1]], dtype=np.int32)
    elif case == "p0_h_layer_only":
        p = 0
    elif case == "k1_single":
        K = 1
    elif case == "gamma_one":
        kw = dict(p1=0.05, p2=0.1, damping=1.0)
    elif case == "full_depolarizing":
        kw = dict(p1=0.75, p2=15 / 16, damping=0.0)
    elif case == "product_mode":
        kw = dict(p1=0.05, p2=0.2, damping=0.05, twoq_mode=1)
    elif case == "lambda_param":
        kw = dict(p1=0.1, p2=0.2, damping=0.0, param=1)
    elif case == "reversed_edges":
        edges = np.array([[3, 0], [4, 1], [2, 4], [1, 0], [3, 2]], dtype=np.int32)
    elif case == "no_noise":
        kw = dict(p1=0.0, p2=0.0, damping=0.0)
    elif case == "n12_two_tiles":
        n, K = 12, 6
    if edges is None:
        edges = W.ring_graph(n)
    g, b = W.angles(p, 99)
    w = W.Workload(case, n, edges, p, g, b, kw.get("p1", 0.0), kw.get("p2", 0.0), kw.get("damping", 0.0), K, K,
                   1234 + n, kw.get("twoq_mode", 0), kw.get("param", 0))
    gpu = run_gpu(qn, w)
    orc, gates, G, nz = run_oracle(w)
    compare_trajectories(gpu, orc, w, G, allow_damp_mismatch=0)
    np.testing.assert_allclose(gpu["probs"], orc["probs_sum"] / K, atol=2e-6)
    assert abs(gpu["mean"] - orc["s1"] / K) < TOL_CT


def test_full_size_damping_n20_sampled(qn):
    """The 20-qubit p=3 damping workload at full size (K=4096, 64 per launch):
    sampled trajectories against the oracle one by one, plus properties."""
    w = W.damping_n20()
    b = qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch)
    b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
    mean, se = b.expectation()
    probs = b.probs()
    assert abs(probs.sum() - 1) < 1e-5
    assert np.all(probs >= 0)
    assert 0 < mean < len(w.edges) and 0 < se < 1
    ids = [0, 1, 63, 64, 2049, 4095]
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    for t in ids:
        dbg = b.traj_debug(t, 1)
        orc = oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, t, 1)
        compare_trajectories(dict(branches=dbg["branches"], amps=dbg["amps"], c_traj=dbg["c_traj"]), orc, w, G)
    info = b.run_info()
    assert info["gates"] == G == 170
    b.close()


def test_deterministic_and_batch_independent(qn):
    """Same seed -> bit-identical results; the launch batch size changes neither a
    trajectory's result nor S1 (accumulated in trajectory order)."""
    w = W.qaoa_workload("det", 12, 2, index=3, trajectories=40, batch=40, damping=0.02)
    r1 = run_gpu(qn, w, launch_batch=40)
    r2 = run_gpu(qn, w, launch_batch=40)
    r3 = run_gpu(qn, w, launch_batch=7)
    assert r1["mean"] == r2["mean"] and np.array_equal(r1["probs"], r2["probs"])
    np.testing.assert_array_equal(r1["branches"], r3["branches"])
    np.testing.assert_array_equal(r1["c_traj"], r3["c_traj"])
    np.testing.assert_array_equal(r1["amps"], r3["amps"])
    assert r1["mean"] == r3["mean"]
    np.testing.assert_allclose(r1["probs"], r3["probs"], atol=1e-7)


def test_invalid_inputs(qn):
    import ctypes
    b = qn.Batch(4, 8, 1)
    with pytest.raises(qn.QnError, match="QN_ESTATE"):
        b.expectation()
    bad = [dict(edges=[[0, 4]]), dict(edges=[[1, 1]]), dict(edges=[[0, 1], [1, 0]])]
    for kw in bad:
        with pytest.raises(qn.QnError, match="QN_EINVAL"):
            b.run_qaoa(kw["edges"], [0.1], [0.2])
    for nzkw in (dict(p1=1.5), dict(p2=-0.1), dict(damping=1.2), dict(twoq_mode=3), dict(param=2),
                 dict(p1=1.4, param=1)):
        with pytest.raises(qn.QnError, match="QN_EINVAL"):
            b.run_qaoa([[0, 1]], [0.1], [0.2], **nzkw)
    b.run_qaoa([[0, 1]], [0.1], [0.2], p1=0.01)
    out = np.zeros(8)
    assert qn.qn_probs(b._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 8) == qn.QN_EINVAL
    # sigma into a caller's buffer, reused across reads
    buf = np.full(16, np.nan)
    assert b.probs(out=buf) is buf and np.array_equal(buf, b.probs())
    for bad in (np.zeros(16, dtype=np.float32), np.zeros(8), np.zeros(32)[::2]):
        with pytest.raises(ValueError):
            b.probs(out=bad)
    with pytest.raises(qn.QnError, match="QN_EINVAL"):
        b.traj_debug(5, 4)
    b.close()

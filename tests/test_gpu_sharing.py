"""Shared-prefix mode (qn_batch_set_sharing): trajectories share the state of
their common Kraus prefix and fork when their own draws diverge.

Exactness checks: the number of distinct states equals the number of distinct
full Kraus strings among the trajectories (from the one-by-one re-simulation),
and the ensemble results equal the default mode's up to FP summation order and
the oracle's within the FP32 bound."""
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


def run(qn, w, sharing, launch_batch=0, fusion=False):
    """fusion=False: one sweep per gate (with Pauli-only noise fusion would take
    precedence over sharing); fusion=True with damping: phase-gate groups."""
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=launch_batch) as b:
        b.set_sharing(sharing)
        b.set_fusion(fusion)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, se = b.expectation()
        probs = b.probs()
        info = b.run_info()
        br = b.traj_debug(0, w.trajectories, amps=False, c=False)["branches"] if sharing else None
    return mean, se, probs, info, br


CASES = {
    "n8_pauli": dict(n=8, p=1, index=0, trajectories=1024, p1=1e-3, p2=1e-2, damping=0.0),
    "n12_damping": dict(n=12, p=2, index=31, trajectories=300, p1=5e-3, p2=2e-2, damping=0.02),
    "n14_damping_multitile": dict(n=14, p=2, index=32, trajectories=96, p1=1e-2, p2=3e-2, damping=0.05),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_sharing_equals_default_mode_and_oracle(qn, case):
    kw = dict(CASES[case])
    n, p, idx, K = kw.pop("n"), kw.pop("p"), kw.pop("index"), kw.pop("trajectories")
    w = W.qaoa_workload(case, n, p, index=idx, trajectories=K, batch=K, **kw)
    m1, s1, p1, _, _ = run(qn, w, False)
    m2, s2, p2, info, br = run(qn, w, True)
    distinct = len({bytes(r) for r in br})
    assert info["states"] == distinct  # one shared state per distinct Kraus string
    if case != "n14_damping_multitile":  # heavy noise: every string differs there
        assert distinct < K
    assert abs(m1 - m2) < 1e-9 and abs(s1 - s2) < 1e-9
    assert abs(p1.sum() - 1) < 1e-12 and abs(p2.sum() - 1) < 1e-12
    np.testing.assert_allclose(p2, p1, rtol=1e-12, atol=0)
    assert abs(oracle.error(p2, p1)) < 1e-12
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, K,
                          want_amps=False, want_branches=False)
    assert abs(m2 - ref["s1"] / K) < TOL_MEAN
    assert oracle.error(p2, ref["probs_sum"] / K) < 1e-9


def test_sharing_in_chunks_and_with_offset(qn):
    """K larger than the launch batch: chunks of 37 trajectories form their own
    prefix trees; a nonzero global offset selects other Philox streams."""
    w = W.qaoa_workload("chunks", 10, 2, index=33, trajectories=100, batch=37, p1=5e-3, p2=2e-2, damping=0.03)
    res = []
    for sharing in (False, True):
        with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=37) as b:
            b.set_sharing(sharing)
            b.set_fusion(False)
            b.set_offset(1000)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            res.append((b.expectation(), b.probs()))
    (ma, _), pa = res[0]
    (mb, _), pb = res[1]
    assert abs(ma - mb) < 1e-9
    np.testing.assert_allclose(pa, pb, atol=1e-12)


@pytest.mark.parametrize("n,K,noise", [
    (12, 1, dict(p1=1e-2, p2=3e-2, damping=0.05)),   # one state through every group
    (12, 2, dict(p1=0.2, p2=0.4, damping=0.1)),      # forks at nearly every group, the last block too
    (16, 5, dict(p1=5e-3, p2=2e-2, damping=0.02)),   # more tile bits, a ragged chunk of states
])
def test_grouped_mode_tiny_ensembles(qn, n, K, noise):
    """Shared prefixes with phase groups and mixer blocks on a handful of trajectories:
    the last block swept for its norms only and applied again by the sigma pass, with
    one state, forks at the last block, and short chunks."""
    w = W.qaoa_workload(f"tiny_n{n}_K{K}", n, 1, index=50 + K, trajectories=K, batch=K, **noise)
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_fusion(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, _ = b.expectation()
        probs = b.probs()
        info = b.run_info()
        br = b.traj_debug(0, K, amps=False, c=False)["branches"]
    assert info["states"] == len({bytes(r) for r in br})
    assert abs(probs.sum() - 1) < 1e-12 and np.all(probs >= 0)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, K,
                          want_amps=False)
    assert np.any(br != ref["branches"], axis=1).sum() == 0
    assert abs(mean - ref["s1"] / K) < TOL_MEAN
    assert oracle.error(probs, ref["probs_sum"] / K) < 1e-9


@pytest.mark.parametrize("n", [26, 28])
def test_grouped_mode_large_n_against_per_gate_sweeps(qn, n):
    """Large states (512 MiB and 2 GiB; n=26 ends on a partial mixer block whose sweep
    stores the states, n=28 on a full one swept for its norms only): the grouped mode
    against one sweep per gate in shared-prefix mode (itself checked against the oracle
    at smaller n) on the same draws -- the same distinct states, <C> within the FP32
    bound, sigma to FP32 state rounding, and sum(sigma) = 1 to FP64 rounding."""
    w = W.qaoa_workload(f"grouped_n{n}", n, 1, index=60, trajectories=6, batch=6, p1=5e-3, p2=3e-2, damping=0.03)
    out = {}
    for fusion in (False, True):
        with qn.Batch(w.n, w.trajectories, w.seed) as b:
            b.set_sharing(True)
            b.set_fusion(fusion)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            out[fusion] = (b.expectation()[0], b.probs(), b.run_info())
    (m1, p1, i1), (m2, p2, i2) = out[False], out[True]
    assert i1["states"] == i2["states"]
    assert i2["sweep_bytes"] < 0.5 * i1["sweep_bytes"]
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    assert abs(m2 - m1) < TOL_CT
    assert abs(p1.sum() - 1) < 1e-12 and abs(p2.sum() - 1) < 1e-12
    assert np.abs(p2 - p1).max() < 1e-6
    assert oracle.error(p2, p1) < 1e-9


def test_bench_mode_full_size_sample_against_oracle(qn):
    """The bench's mode (shared prefixes, phase groups, 4-qubit mixer blocks; the last
    block swept for its norms only and applied again by the sigma pass) on the 20-qubit
    p=3 damping circuit, for a sample of 48 trajectories (global ids 2000..2047) that the
    oracle evolves one by one: the ensemble <C>, sigma and the number of distinct states."""
    w = W.damping_n20()
    K, t0 = 48, 2000
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_fusion(True)
        b.set_offset(t0)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, _ = b.expectation()
        probs = b.probs()
        info = b.run_info()
        br = b.traj_debug(0, K, amps=False, c=False)["branches"]
    assert info["states"] == len({bytes(r) for r in br})
    assert abs(probs.sum() - 1) < 1e-12 and np.all(probs >= 0)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, t0, K,
                          want_amps=False)
    np.testing.assert_array_equal(br & 15, ref["branches"] & 15)  # Pauli codes: bit-exact
    # damping branches may differ only where u lies within FP32 reach of p1 (counted)
    assert np.any(br != ref["branches"], axis=1).sum() <= 1
    assert abs(mean - ref["s1"] / K) < TOL_MEAN
    assert oracle.error(probs, ref["probs_sum"] / K) < 1e-9


def test_sharing_full_size_damping_n20(qn):
    """The 20-qubit p=3 damping workload (K=4096) in shared-prefix mode against
    the default mode."""
    w = W.damping_n20()
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        m1, s1 = b.expectation()
        p1 = b.probs()
    out = {}
    for fusion in (False, True):  # one sweep per gate / phase gates in groups
        with qn.Batch(w.n, w.trajectories, w.seed) as b:
            b.set_sharing(True)
            b.set_fusion(fusion)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            out[fusion] = (b.expectation(), b.probs(), b.run_info())
    (m2, s2), p2, info2 = out[False]
    (m3, s3), p3, info3 = out[True]
    assert info2["states"] < w.trajectories and info3["states"] == info2["states"]
    assert abs(m1 - m2) < 1e-8 and abs(s1 - s2) < 1e-8
    np.testing.assert_allclose(p2, p1, rtol=1e-12, atol=0)
    G = w.gate_count
    assert abs(m3 - m1) < TOL_MEAN
    assert np.abs(p3 - p1).max() < 1e-6
    assert info3["sweep_bytes"] < 0.7 * info2["sweep_bytes"]


GROUP_CASES = {
    "n5_ring_partial_warp": dict(n=5, p=2, index=40, trajectories=200, p1=5e-3, p2=2e-2, damping=0.03, d=2),
    "n12_damping": dict(n=12, p=2, index=31, trajectories=300, p1=5e-3, p2=2e-2, damping=0.02),
    "n14_heavy_noise": dict(n=14, p=2, index=32, trajectories=96, p1=1e-2, p2=3e-2, damping=0.05),
    "n16_d5_ragged_groups": dict(n=16, p=1, index=41, trajectories=400, p1=2e-3, p2=1e-2, damping=0.01, d=5),
    # 18 edges on 9 qubits: phase groups end at the 12-gate limit
    "n9_d4_gate_limit": dict(n=9, p=2, index=42, trajectories=300, p1=5e-3, p2=2e-2, damping=0.02, d=4),
    # mixer blocks of 4, 4, 4 and 1 qubits: the last one takes the generic sweep
    "n13_d4_one_qubit_block": dict(n=13, p=2, index=43, trajectories=200, p1=5e-3, p2=2e-2, damping=0.02, d=4),
}


@pytest.mark.parametrize("case", sorted(GROUP_CASES))
def test_phase_groups_equal_per_gate_sharing_and_oracle(qn, case):
    """Shared-prefix mode with damping, phase gates swept in groups (one joint
    per group, one apply sweep) against the per-gate shared-prefix run, the
    default mode and the oracle.  The Kraus strings are the same draws, so the
    number of distinct states must match exactly."""
    kw = dict(GROUP_CASES[case])
    n, p, idx, K = kw.pop("n"), kw.pop("p"), kw.pop("index"), kw.pop("trajectories")
    w = W.qaoa_workload(case, n, p, index=idx, trajectories=K, batch=K, **kw)
    m0, s0, p0, _, _ = run(qn, w, False)
    m1, s1, p1, info1, br = run(qn, w, True, fusion=False)
    m2, s2, p2, info2, _ = run(qn, w, True, fusion=True)
    distinct = len({bytes(r) for r in br})
    assert info1["states"] == distinct and info2["states"] == distinct
    assert info2["sweep_bytes"] < info1["sweep_bytes"]  # fewer sweeps over the states
    # same draws: the ensemble sums agree to FP32 state rounding
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    tol = TOL_MEAN
    assert abs(m2 - m1) < tol and abs(m2 - m0) < tol
    assert abs(p2.sum() - 1) < 1e-12
    assert np.abs(p2 - p0).max() < 1e-5
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, K,
                          want_amps=False, want_branches=False)
    assert abs(m2 - ref["s1"] / K) < tol
    assert oracle.error(p2, ref["probs_sum"] / K) < 1e-9


def test_phase_groups_deterministic_and_chunked(qn):
    """Two runs give bit-identical results (joints are summed in a fixed order);
    chunks of 37 trajectories with an offset agree with the default mode."""
    w = W.qaoa_workload("grp_chunks", 10, 2, index=33, trajectories=100, batch=37, p1=5e-3, p2=2e-2, damping=0.03)
    res = []
    for sharing in (False, True, True):
        with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=37) as b:
            b.set_sharing(sharing)
            b.set_offset(1000)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            res.append((b.expectation(), b.probs()))
    (ma, _), pa = res[0]
    (mb, sb), pb = res[1]
    (mc, sc), pc = res[2]
    assert mb == mc and sb == sc and np.array_equal(pb, pc)
    assert abs(ma - mb) < 1e-5
    assert np.abs(pa - pb).max() < 1e-5

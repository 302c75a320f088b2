"""Element-by-element parity of the shared-prefix path -- the bench's own kernels --
with the FP64 oracle (O2), read out of the run itself (qn_shared_readout): no
re-simulation.  Per trajectory: the Kraus string the run drew (the group decide's
draws with phase groups and mixer blocks; the slot decide's gate by gate), <C>_t as
the sigma pass formed it, and the final state (a pending last mixer block applied
to the slot's stored state with its drawn factors).  Ensemble: sigma element by
element and the mean <C>.

Bars (derivations in the docstrings of the helpers):
  * Pauli codes bit-exact;
  * damping strings equal, except where the draw u lies within FP32 reach of the
    branch probability (the group decide draws in FP32): counted, at most one per
    case; such a trajectory is compared with the oracle's state along the GPU's
    own (valid, nonzero-weight) string;
  * amplitudes within 1e-5 absolute;
  * <C>_t within TOL_CT = 2e-5 absolute, the ensemble mean within 2e-6;
  * sigma_x within 2e-5 relative (plus 1e-12 absolute) of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_AMP = 1e-5
TOL_CT = 2e-5
TOL_MEAN = 2e-6
RTOL_SIGMA = 2e-5


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


def reference_states(w, orc, gpu_br, gates, G, nz):
    """The oracle's final states, except that a trajectory whose damping string differs
    from the GPU's is replaced by the oracle's state along the GPU's string (forced
    branches): such a string must have nonzero Born weight, and the GPU state must
    match it.  Returns (states [K, 2^n], number of replaced trajectories)."""
    ref = orc["amps"].copy()
    diff = np.where(np.any(gpu_br != orc["branches"], axis=1))[0]
    for t in diff:
        psi, weight = oracle.traj_forced(w.n, gates, G, nz, gpu_br[t])
        assert psi is not None and weight > 0.0, f"trajectory {t}: the GPU's string has zero weight"
        ref[t] = psi
    return ref, len(diff)


def check_members(w, gpu, orc, gates, G, nz, max_mismatch=1):
    """Per-trajectory parity; returns the measured errors."""
    br = gpu["branches"]
    np.testing.assert_array_equal(br & 15, orc["branches"] & 15)  # Pauli codes: bit-exact
    ref, nmis = reference_states(w, orc, br, gates, G, nz)
    assert nmis <= max_mismatch, f"{nmis} damping-string mismatches"
    amp_err = float(np.abs(gpu["amps"] - ref).max())
    assert amp_err < TOL_AMP, amp_err
    cut = oracle.cut_values(w.n, w.edges)
    c_ref = (np.abs(ref) ** 2) @ cut
    ct_err = float(np.abs(gpu["c_traj"] - c_ref).max())
    assert ct_err < TOL_CT, ct_err
    return dict(mismatches=nmis, amp_err=amp_err, ct_err=ct_err, ref=ref, c_ref=c_ref)


CASES = {
    # n, p, index, K, noise, degree; comments: how the circuit ends
    "n12_keep_last_block": (12, 3, 70, 1024, dict(p1=5e-3, p2=2e-2, damping=0.02), 3),  # last block pending
    "n14_partial_last_block": (14, 2, 71, 512, dict(p1=1e-2, p2=3e-2, damping=0.05), 3),  # 2-qubit block stored
    "n16_bench_noise": (16, 3, 72, 512, dict(p1=1e-3, p2=1e-2, damping=5e-3), 3),  # last block pending
    "n13_one_qubit_block": (13, 2, 73, 400, dict(p1=5e-3, p2=2e-2, damping=0.02), 4),  # generic last block
    "n9_per_gate_mixers": (9, 2, 74, 600, dict(p1=5e-3, p2=2e-2, damping=0.03), 4),  # mixer gates one by one
    # mixer blocks 0-7 (rotated whole by the last phase group's sweep), 8-15 (over two sweeps),
    # 16-19; heavy noise so that slots fork at every block
    "n20_split8_blocks": (20, 2, 75, 16, dict(p1=3e-2, p2=8e-2, damping=0.05), 3),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("fusion", [True, False], ids=["groups", "per_gate"])
def test_shared_prefix_states_against_oracle(qn, case, fusion):
    n, p, idx, K, noise, d = CASES[case]
    w = W.qaoa_workload(case, n, p, index=idx, trajectories=K, batch=K, d=d, **noise)
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_fusion(fusion)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, _ = b.expectation()
        sigma = b.probs()
        info = b.run_info()
        gpu = b.shared_readout(0, K)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    orc = oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, 0, K)
    # one state per distinct Kraus string that the run itself drew
    assert info["states"] == len({bytes(r) for r in gpu["branches"]})
    res = check_members(w, gpu, orc, gates, G, nz)
    # the ensemble: <C> and sigma element by element
    assert abs(mean - res["c_ref"].mean()) < TOL_MEAN
    assert abs(mean - gpu["c_traj"].mean()) < 1e-12  # S1 sums exactly the <C>_t read out
    sig_ref = (np.abs(res["ref"]) ** 2).sum(axis=0) / K
    np.testing.assert_allclose(sigma, sig_ref, rtol=RTOL_SIGMA, atol=1e-12)
    assert abs(sigma.sum() - 1) < 1e-12
    print(f"{case} fusion={fusion}: states {info['states']}, mismatches {res['mismatches']}, "
          f"max |d amp| {res['amp_err']:.2e}, max |d <C>_t| {res['ct_err']:.2e}, "
          f"|d mean| {abs(mean - res['c_ref'].mean()):.2e}, "
          f"max rel d sigma {np.max(np.abs(sigma - sig_ref) / np.maximum(sig_ref, 1e-300)):.2e}")


def test_bench_mode_full_ensemble_against_oracle_and_per_trajectory_path(qn):
    """The bench's own run (n=20, p=3, depolarizing + damping, K=4096, shared prefixes
    with phase groups and mixer blocks 0-7, 8-15, 16-19, the last block pending): trajectories
    2000..2047 of that run against the oracle, member by member (amplitudes for
    2000..2015); and the Kraus strings of all 4096 trajectories against the
    one-state-per-trajectory path (FP64 draws gate by gate): Pauli codes bit-exact,
    damping-string mismatches counted (FP32 edge cases of the group decide)."""
    w = W.damping_n20()
    K, s0, ns, na = w.trajectories, 2000, 48, 16
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_fusion(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, se = b.expectation()
        info = b.run_info()
        allbr = b.shared_readout(0, K, amps=False, c=False)["branches"]
        part = b.shared_readout(s0, ns, amps=False)
        amps = b.shared_readout(s0, na, branches=False, c=False)["amps"]
        per_traj = b.traj_debug(0, K, amps=False, c=False)["branches"]  # re-simulates one by one
    assert info["states"] == len({bytes(r) for r in allbr})
    np.testing.assert_array_equal(allbr & 15, per_traj & 15)
    mism = int(np.any(allbr != per_traj, axis=1).sum())
    print(f"n=20 K=4096: {info['states']} states, {mism} damping-string mismatches against the "
          f"per-trajectory path")
    assert mism <= 2
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    orc = oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, s0, ns, want_amps=False)
    np.testing.assert_array_equal(part["branches"] & 15, orc["branches"] & 15)
    same = np.all(part["branches"] == orc["branches"], axis=1)
    assert (~same).sum() <= 1
    ct_err = float(np.abs(part["c_traj"][same] - orc["c_traj"][same]).max())
    assert ct_err < TOL_CT, ct_err
    orc_a = oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, s0, na)
    ref, nmis = reference_states(w, orc_a, part["branches"][:na], gates, G, nz)
    amp_err = float(np.abs(amps - ref).max())
    assert amp_err < TOL_AMP, amp_err
    print(f"n=20 sample: max |d amp| {amp_err:.2e}, max |d <C>_t| {ct_err:.2e}, <C> = {mean:.6f} +- {se:.6f}")


def test_shared_readout_rejects_what_it_cannot_read(qn):
    w = W.qaoa_workload("readout_guard", 10, 1, index=75, trajectories=40, batch=40, p1=1e-2, p2=3e-2,
                        damping=0.02)
    with qn.Batch(w.n, w.trajectories, w.seed) as b:
        b.set_sharing(False)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        with pytest.raises(qn.QnError) as e:
            b.shared_readout(0, 4)
        assert e.value.status == qn.QN_ESTATE
        b.set_sharing(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        with pytest.raises(qn.QnError) as e:
            b.shared_readout(30, 20)  # beyond the ensemble
        assert e.value.status == qn.QN_EINVAL
        first = b.shared_readout(0, 40)
        again = b.shared_readout(10, 5)  # reading does not disturb the run's buffers
        np.testing.assert_array_equal(again["amps"], first["amps"][10:15])
        np.testing.assert_array_equal(again["c_traj"], first["c_traj"][10:15])
        b.traj_debug(0, 2)  # re-simulation reuses the buffers: the readout is gone
        with pytest.raises(qn.QnError) as e:
            b.shared_readout(0, 4)
        assert e.value.status == qn.QN_ESTATE


def test_shards_on_two_handles_equal_one_handle(qn):
    """Sample parallelism (Sec. "Parallelism Hierarchy"): two handles on disjoint
    global id ranges, combined by shards.finish, equal one handle over the union
    (every draw is keyed by the global trajectory id) -- in the bench's mode."""
    from paper_2210_15874_gb300 import shards

    w = W.qaoa_workload("shards_n14", 14, 2, index=76, trajectories=700, batch=700, p1=5e-3, p2=2e-2,
                        damping=0.02)
    K = w.trajectories
    parts = []
    for rank in range(2):
        first, count = shards.shard_range(K, 2, rank)
        with qn.Batch(w.n, count, w.seed) as b:
            b.set_sharing(True)
            b.set_fusion(True)
            b.set_offset(first)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            m, s = b.expectation()
            parts.append(shards.local_sums(m, s, b.probs(), count))
    mean, se, sigma = shards.finish(parts[0] + parts[1])
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_fusion(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        m1, s1 = b.expectation()
        p1 = b.probs()
    assert abs(mean - m1) < 1e-9 and abs(se - s1) < 1e-9
    np.testing.assert_allclose(sigma, p1, rtol=1e-6, atol=1e-12)

"""Device-driven launches of the shared-prefix path against the host-sized ones.

Launch mode 1 (qn_batch_set_launch_mode): every sweep is a persistent launch over
the slots the device counts, every decide kernel reads the live-slot count on the
device, and the sigma pass takes its slot order and row blocks from device steps --
the host reads nothing until the run is over.  Mode 2 captures that run in a CUDA
graph and replays it.  Mode 0 (the default) sizes every launch on the host from
the live count it reads after each decide.

The modes launch the same arithmetic on the same draws, so everything a run leaves
is bit-identical across them: each trajectory's Kraus string, final state and <C>_t
(read out of the run itself), sigma (the device chooses the sigma pass's row
blocks from its own count by the host's rule) and the ensemble sums.  Mode 0 is
checked against the FP64 oracle in test_gpu_shared_parity.py; one case here checks
a replayed graph against the oracle directly.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2210_15874_gb300 import workloads as W
from tolerances import TOL_AMP, TOL_CT, TOL_MEAN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


CASES = {
    # n, p, index, K, noise, degree
    "n12_keep_last_block": (12, 3, 70, 1024, dict(p1=5e-3, p2=2e-2, damping=0.02), 3),
    "n14_partial_last_block": (14, 2, 71, 512, dict(p1=1e-2, p2=3e-2, damping=0.05), 3),
    "n13_one_qubit_block": (13, 2, 73, 400, dict(p1=5e-3, p2=2e-2, damping=0.02), 4),
    "n9_per_gate_mixers": (9, 2, 74, 600, dict(p1=5e-3, p2=2e-2, damping=0.03), 4),
    "n20_split8_blocks": (20, 2, 75, 16, dict(p1=3e-2, p2=8e-2, damping=0.05), 3),
    "n5_partial_warp": (5, 2, 77, 300, dict(p1=2e-2, p2=5e-2, damping=0.05), 4),
}


def run(qn, w, mode, *, fusion=True, offset=0, readout=True):
    """One shared-prefix run of workload w in launch mode `mode` (one prefix tree holds
    the whole ensemble at these sizes, so the readout covers every trajectory)."""
    K = w.trajectories
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_fusion(fusion)
        b.set_launch_mode(mode)
        b.set_offset(offset)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        out = dict(stats=b.expectation(), sigma=b.probs(), info=b.run_info())
        if readout:
            out["read"] = b.shared_readout(0, K)
    return out


def assert_same(a, b):
    assert a["stats"] == b["stats"]
    np.testing.assert_array_equal(a["sigma"], b["sigma"])
    assert a["info"]["states"] == b["info"]["states"]
    assert a["info"]["sweep_bytes"] == b["info"]["sweep_bytes"]
    if "read" in a and "read" in b:
        for k in ("branches", "c_traj", "amps"):
            np.testing.assert_array_equal(a["read"][k], b["read"][k])


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("fusion", [True, False], ids=["groups", "per_gate"])
def test_device_driven_runs_equal_host_sized_runs(qn, case, fusion):
    n, p, idx, K, noise, d = CASES[case]
    w = W.qaoa_workload(case, n, p, index=idx, trajectories=K, batch=K, d=d, **noise)
    host = run(qn, w, 0, fusion=fusion)
    dev = run(qn, w, 1, fusion=fusion)
    assert_same(host, dev)
    assert abs(dev["sigma"].sum() - 1.0) < 1e-12


def test_graph_replays_and_updates(qn):
    """Mode 2 on one handle: the first run captures, an identical run replays, a run
    over another trajectory range of the same circuit replays, and a run with other
    angles captures again (updating the instantiated graph in place); each equals a
    host-sized run of the same inputs."""
    n, p, idx, K, noise, d = CASES["n12_keep_last_block"]
    w = W.qaoa_workload("graph_n12", n, p, index=idx, trajectories=K, batch=K, d=d, **noise)
    other = W.qaoa_workload("graph_n12b", n, p, index=idx + 100, trajectories=K, batch=K, d=d, **noise)
    w2 = dataclasses.replace(w, gammas=other.gammas, betas=other.betas)  # same circuit shape, new angles
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_launch_mode(2)
        results = []
        for wk, off in ((w, 0), (w, 0), (w, 5000), (w2, 5000), (w, 0)):
            b.set_offset(off)
            b.run_qaoa(wk.edges, wk.gammas, wk.betas, **wk.noise_kwargs())
            results.append((wk, off, dict(stats=b.expectation(), sigma=b.probs(), info=b.run_info(),
                                          read=b.shared_readout(0, K))))
        gi = b.graph_info()
    assert gi["replays"] >= 2, gi
    assert gi["captures"] + gi["replays"] == 5, gi
    assert gi["captures"] <= 3, gi
    for wk, off, res in results:
        assert_same(run(qn, wk, 0, offset=off), res)
    # the identical runs are identical; the other range is not
    assert results[0][2]["stats"] == results[1][2]["stats"] == results[4][2]["stats"]
    assert results[2][2]["stats"] != results[0][2]["stats"]


def test_replayed_graph_against_oracle(qn):
    """A replayed graph's per-trajectory results against the FP64 oracle (the bars of
    tests/tolerances.py; Pauli codes bit-exact, damping strings equal)."""
    n, p, idx, K, noise, d = CASES["n14_partial_last_block"]
    K = 256
    w = W.qaoa_workload("graph_oracle", n, p, index=idx, trajectories=K, batch=K, d=d, **noise)
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_launch_mode(2)
        for _ in range(2):
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        assert b.graph_info()["replays"] == 1
        mean, _ = b.expectation()
        sigma = b.probs()
        gpu = b.shared_readout(0, K)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    orc = oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, 0, K)
    np.testing.assert_array_equal(gpu["branches"] & 15, orc["branches"] & 15)
    # a damping draw within FP32 reach of its branch probability may go the other way
    # (the group decide draws in FP32): at most one such trajectory, left out below
    same = np.all(gpu["branches"] == orc["branches"], axis=1)
    assert (~same).sum() <= 1
    assert float(np.abs(gpu["amps"][same] - orc["amps"][same]).max()) < TOL_AMP
    assert float(np.abs(gpu["c_traj"][same] - orc["c_traj"][same]).max()) < TOL_CT
    if same.all():
        assert abs(mean - orc["c_traj"].mean()) < TOL_MEAN
        sig_ref = (np.abs(orc["amps"]) ** 2).sum(axis=0) / K
        np.testing.assert_allclose(sigma, sig_ref, rtol=2e-5, atol=1e-12)


def test_bench_workload_in_every_mode(qn):
    """The bench's ensemble (n=20, p=3, K=4096, depolarizing + damping): the device-driven
    run and two runs of its graph equal the host-sized run."""
    w = W.damping_n20()
    K = w.trajectories
    host = run(qn, w, 0, readout=False)
    dev = run(qn, w, 1, readout=False)
    assert_same(host, dev)
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.set_launch_mode(2)
        for _ in range(2):
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            res = dict(stats=b.expectation(), sigma=b.probs(), info=b.run_info())
            assert_same(host, res)
        assert b.graph_info() == dict(captures=1, replays=1, updates=0)
        part = b.shared_readout(2000, 16)
    with qn.Batch(w.n, K, w.seed) as b:
        b.set_sharing(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        ref = b.shared_readout(2000, 16)
    for k in ("branches", "c_traj", "amps"):
        np.testing.assert_array_equal(part[k], ref[k])

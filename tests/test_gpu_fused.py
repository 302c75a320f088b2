"""Fused layers (Pauli-only noise): one sweep per window of up to eight qubits per
QAOA layer instead of one per gate.  Checked against the per-gate sweeps and the FP64 oracle on the
same trajectories: Pauli codes bit-exact, amplitudes within 1e-5, <C>_t within
the FP32 bound; the precision figures at n=14 are printed (pytest -s)."""
import json

import numpy as np
import pytest

import oracle
from tolerances import TOL_CT
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def fused_windows(n):
    """Windows (first qubit, qubits) of one layer of the FP32 fused schedule: below ten
    qubits five at a time (registers only); from ten on the window that holds qubit 0,
    then balanced windows of at most 7 over the rest, larger first (the qubits beyond
    four on lane bits).  The first window is qubits 0-11 (one 2048-float4 tile in
    shared memory) where that leaves fewer windows than qubits 0-7 (qubit 0 in the
    float4, 1-3 on lane bits, 4-7 in registers) does."""
    if n < 10:
        return [(q, min(5, n - q)) for q in range(0, n, 5)]
    first = 12 if n > 12 and -(-(n - 12) // 7) < -(-(n - 8) // 7) else 8
    rest = n - first
    count = -(-rest // 7)
    out, q = [(0, first)], first
    for i in range(count):
        m = rest // count + (1 if i < rest % count else 0)
        out.append((q, m))
        q += m
    return out


def fused_sweeps(n):
    return len(fused_windows(n))


def test_fused_windows_cover_each_qubit_once():
    for n in range(2, 33):
        w = fused_windows(n)
        assert [q for lo, m in w for q in range(lo, lo + m)] == list(range(n))
        assert all(m <= (7 if n >= 10 else 5) for _, m in w[1:])
    assert [fused_sweeps(n) for n in (14, 16, 20, 24, 26, 30)] == [2, 2, 3, 3, 3, 4]
    assert [fused_windows(n)[0][1] for n in range(13, 32)] == \
        [8, 8, 8, 12, 12, 12, 12, 8, 8, 8, 12, 12, 12, 12, 8, 8, 8, 12, 12]


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


def run(qn, w, fusion, launch_batch=0):
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=launch_batch) as b:
        b.set_fusion(fusion)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, se = b.expectation()
        probs = b.probs()
        dbg = b.traj_debug(0, w.trajectories)
        info = b.run_info()
    return dict(mean=mean, se=se, probs=probs, info=info, **dbg)


# every window form: registers only (n < 10, and the 2-4-qubit windows after qubit 7 or 11),
# qubits 0-7 with three lane qubits (n >= 10), 5, 6, 7-qubit windows with one, two,
# three lane qubits (n = 13, 14, 15, 19), and the 12-qubit tile (n = 16: 12 + 4, 16 tiles
# per state; n = 17: 12 + 5; n = 19: 12 + 7)
@pytest.mark.parametrize("n,p,edges_kind", [(2, 1, "one"), (3, 2, "ring"), (4, 2, "ring"), (7, 2, "reg"),
                                            (8, 1, "reg"), (10, 2, "reg"), (12, 3, "reg"), (13, 2, "reg"),
                                            (14, 2, "reg"), (15, 2, "reg"), (16, 2, "reg"), (17, 1, "reg"),
                                            (19, 1, "reg")])
def test_fused_matches_per_gate_and_oracle(qn, n, p, edges_kind):
    if edges_kind == "one":
        edges = np.array([[0, 1]], dtype=np.int32)
    elif edges_kind == "ring":
        edges = W.ring_graph(n)
    else:
        edges = W.regular_graph(n, 3 if n % 2 == 0 else 4, 70 + n)
    g, b = W.angles(p, 80 + n)
    K = 24
    w = W.Workload(f"fused_n{n}", n, edges, p, g, b, 0.02, 0.05, 0.0, K, K, 555 + n)
    fused = run(qn, w, True, launch_batch=10)
    plain = run(qn, w, False, launch_batch=10)
    gates, G = oracle.qaoa_gates(n, edges, g, b)
    ref = oracle.traj_run(n, edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, K)
    np.testing.assert_array_equal(fused["branches"], ref["branches"])
    tol_c = TOL_CT
    for res in (fused, plain):
        assert np.abs(res["amps"] - ref["amps"]).max() < 1e-5
        assert np.abs(res["c_traj"] - ref["c_traj"]).max() < tol_c
        assert abs(res["mean"] - ref["s1"] / K) < tol_c
    assert np.abs(fused["amps"] - plain["amps"]).max() < 1e-5
    # fewer sweeps: launches per batch = prepare + init + p layer-parameter kernels
    # + p fused sweeps per layer + the norm pass (folded into the last sweep when
    # that window is off qubit 0, n > 5) + probs
    nb = -(-K // 10)
    assert fused["info"]["launches"] == nb * (2 + p + p * fused_sweeps(n) + (1 if n <= 5 else 0) + 1)


def test_fused_precision_n14(qn):
    """The 26/30-qubit precision workload's circuit family (3-regular, p=4,
    p1=1e-3, p2=1e-2) at n=14 against the FP64 oracle, both schedules."""
    w = W.qaoa_workload("precision_n14", 14, 4, index=2, trajectories=32, batch=32)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, w.trajectories)
    out = {}
    for name, fusion in (("fused", True), ("per_gate", False)):
        r = run(qn, w, fusion)
        d = r["amps"] - ref["amps"]
        out[name] = {"max_abs_amp_err": float(np.abs(d).max()),
                     "rms_amp_err": float(np.sqrt(np.mean(np.abs(d) ** 2))),
                     "max_abs_c_err": float(np.abs(r["c_traj"] - ref["c_traj"]).max()),
                     "mean_c_err": float(abs(r["mean"] - ref["s1"] / w.trajectories)),
                     "sweeps_per_trajectory": int(r["info"]["sweep_bytes"] / (16 * 2 ** w.n * w.trajectories))}
        assert out[name]["max_abs_amp_err"] < 1e-5
    print(json.dumps({"precision_n14_fp32": out, "gates": G}))


def test_fused_at_size_n24_sampled_against_oracle(qn):
    """The precision workload's fused path at a size whose states (128 MiB each) are far
    above L2 and whose tiles cover every mixer-sweep variant: n=24, p=4, 3-regular,
    depolarizing p1=1e-3 / p2=1e-2, two trajectories of a 64-trajectory ensemble
    (global ids 37 and 38) read back from the fused sweeps and compared with the oracle
    amplitude by amplitude.  (n=26 costs the oracle about four minutes per trajectory
    on the host cores; n=24 about one.)"""
    w = W.qaoa_workload("precision_n24", 24, 4, index=2, trajectories=64, batch=16)
    t0, cnt = 37, 2
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
        b.set_fusion(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        info = b.run_info()
        dbg = b.traj_debug(t0, cnt)
    E = len(w.edges)
    assert info["sweep_bytes"] == 16.0 * 2 ** w.n * w.trajectories * w.p * fused_sweeps(w.n)  # fused schedule
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, t0, cnt,
                          threads=cnt)
    np.testing.assert_array_equal(dbg["branches"], ref["branches"])
    err = float(np.abs(dbg["amps"] - ref["amps"]).max())
    c_err = float(np.abs(dbg["c_traj"] - ref["c_traj"]).max())
    print(json.dumps({"fused_n24": {"max_abs_amp_err": err, "max_abs_c_err": c_err, "E": E}}))
    assert err < 1e-5
    assert c_err < 2e-5


def test_fused_tiled_windows_n22_sampled_against_oracle(qn):
    """n=22, p=2 (3-regular, depolarizing p1=2e-2 / p2=5e-2): windows (0, 8), (8, 7), (15, 7), so the
    tiled sweep of a 7-qubit window runs in all three forms -- plain (qubits 8-14), with the next
    layer's phase (qubits 15-21, layer 0) and with the final norms (layer 1).  Two trajectories of an
    8-trajectory ensemble (global ids 3 and 4) against the oracle, amplitude by amplitude."""
    w = W.qaoa_workload("fused_n22", 22, 2, index=5, trajectories=8, batch=8, p1=2e-2, p2=5e-2)
    assert fused_windows(22) == [(0, 8), (8, 7), (15, 7)]
    t0, cnt = 3, 2
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
        b.set_fusion(True)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        info = b.run_info()
        dbg = b.traj_debug(t0, cnt)
    assert info["sweep_bytes"] == 16.0 * 2 ** w.n * w.trajectories * w.p * 3
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, t0, cnt,
                          threads=cnt)
    np.testing.assert_array_equal(dbg["branches"], ref["branches"])
    err = float(np.abs(dbg["amps"] - ref["amps"]).max())
    c_err = float(np.abs(dbg["c_traj"] - ref["c_traj"]).max())
    print(json.dumps({"fused_n22": {"max_abs_amp_err": err, "max_abs_c_err": c_err}}))
    assert err < 1e-5
    assert c_err < 2e-5

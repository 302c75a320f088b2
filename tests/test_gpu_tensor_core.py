"""The fused layers on the tensor cores (qn_batch_set_precision): five-qubit
windows of mixer rotations as two GEMMs with the +-1 Hadamard matrix
(tcgen05.mma, FP32 accumulation in TMEM), TF32 or BF16x3 split operands.

Checked against the FP64 oracle on the same trajectories (the Kraus draws do not
depend on the arithmetic):
  * Pauli codes bit-exact;
  * BF16x3 (exact products, FP32 accumulation): amplitudes within TOL_AMP = 1e-5
    and <C>_t within TOL_CT, like the FP32 paths;
  * TF32 (10 explicit mantissa bits, u <= 2^-10 per operand whether the hardware
    rounds or truncates): each GEMM's operand rounding perturbs a 32-amplitude
    fiber by at most u times its 2-norm, and the rest of the sweep (H5 / sqrt(32),
    the phases) is unitary, so after S sweeps (two GEMMs each) the state is off by
    at most 2 u S in 2-norm: amplitudes within 2 u S, <C>_t within 2 * 2 u S * E
    (|d<psi|C|psi>| <= 2 ||d psi|| ||C||, ||C|| <= E);
and the precision figures at n=14 (p=4, the precision workload's family) are
printed (pytest -s) for FP32, TF32 and BF16x3.
"""
import json

import numpy as np
import pytest

import oracle
from tolerances import TOL_AMP, TOL_CT
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TF32_U = 2.0 ** -10


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


def run(qn, w, precision, launch_batch=0):
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=launch_batch) as b:
        b.set_fusion(True)
        b.set_precision(precision)
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        mean, se = b.expectation()
        probs = b.probs()
        dbg = b.traj_debug(0, w.trajectories)
        info = b.run_info()
    return dict(mean=mean, se=se, probs=probs, info=info, **dbg)


def sweeps(n, p):
    return p * -(-n // 5)


# windows: n=11 one tile per state and a one-qubit last window; n=12..14 ragged last windows
# below bit 6; n=16, 17 windows above bit 6 with tile bits on both sides
CASES = [(11, 2), (12, 3), (13, 2), (14, 2), (16, 2), (17, 1)]


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
def test_tensor_core_layers_against_oracle(qn, n, p, precision):
    edges = W.regular_graph(n, 3 if n % 2 == 0 else 4, 90 + n)
    g, b = W.angles(p, 95 + n)
    K = 12
    w = W.Workload(f"tc_n{n}", n, edges, p, g, b, 0.02, 0.05, 0.0, K, K, 777 + n)
    res = run(qn, w, precision, launch_batch=5)
    gates, G = oracle.qaoa_gates(n, edges, g, b)
    ref = oracle.traj_run(n, edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, K)
    np.testing.assert_array_equal(res["branches"], ref["branches"])
    S = sweeps(n, p)
    assert res["info"]["sweep_bytes"] == 16.0 * 2 ** n * K * S
    amp_err = float(np.abs(res["amps"] - ref["amps"]).max())
    c_err = float(np.abs(res["c_traj"] - ref["c_traj"]).max())
    if precision == "bf16x3":
        amp_tol, c_tol = TOL_AMP, TOL_CT
    else:
        amp_tol = 2 * TF32_U * S
        c_tol = 4 * TF32_U * S * len(edges)
    print(f"tc n={n} p={p} {precision}: max |d amp| {amp_err:.2e} (bound {amp_tol:.1e}), "
          f"max |d <C>_t| {c_err:.2e} (bound {c_tol:.1e})")
    assert amp_err < amp_tol
    assert c_err < c_tol
    assert abs(res["probs"].sum() - 1) < 1e-6


def test_tensor_core_precision_n14(qn):
    """The precision workload's circuit family (3-regular, p=4, p1=1e-3, p2=1e-2) at
    n=14: each arithmetic against the FP64 oracle, amplitude by amplitude."""
    w = W.qaoa_workload("precision_n14", 14, 4, index=2, trajectories=32, batch=32)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    ref = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, w.trajectories)
    out = {}
    for precision in ("fp32", "tf32", "bf16x3"):
        r = run(qn, w, precision)
        d = r["amps"] - ref["amps"]
        out[precision] = {"max_abs_amp_err": float(np.abs(d).max()),
                          "rms_amp_err": float(np.sqrt(np.mean(np.abs(d) ** 2))),
                          "max_abs_c_err": float(np.abs(r["c_traj"] - ref["c_traj"]).max()),
                          "mean_c_err": float(abs(r["mean"] - ref["s1"] / w.trajectories)),
                          "sweeps_per_trajectory": int(r["info"]["sweep_bytes"] / (16 * 2 ** w.n * w.trajectories))}
    print(json.dumps({"precision_n14": out, "gates": G}))
    assert out["bf16x3"]["max_abs_amp_err"] < TOL_AMP and out["fp32"]["max_abs_amp_err"] < TOL_AMP
    assert out["tf32"]["max_abs_c_err"] < 4 * TF32_U * 12 * len(w.edges)
    # tensor cores: five-qubit windows (3 per layer at n=14); FP32: qubits 0-7 and 8-13 (2 per layer)
    assert out["bf16x3"]["sweeps_per_trajectory"] == 12 and out["fp32"]["sweeps_per_trajectory"] == 8


def test_precision_mode_validation(qn):
    w = W.qaoa_workload("prec_guard", 8, 1, index=3, trajectories=4, batch=4)
    with qn.Batch(w.n, 4, w.seed) as b:
        with pytest.raises(qn.QnError):
            b.set_precision(3)
        b.set_precision("bf16x3")  # below 11 qubits the FP32 fused layers run
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        assert b.run_info()["sweep_bytes"] == 16.0 * 2 ** w.n * 4 * w.p * 2  # qubits 0-4, 5-7 (FP32)

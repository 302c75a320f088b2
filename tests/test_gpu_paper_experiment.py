"""The paper's experiment (Sec. "Results", Eq. 2) rerun on the GPU path.

QAOA p=2 on seeded 4-regular graphs, depolarizing noise with the paper's
lambda parameterisation (lambda1 = 1e-3 after 1q gates, lambda2 = 4e-3 after 2q
gates), ensembles of K = 10 .. 1780 circuits, Error = 1 - F(sigma_approx,
sigma_exact) against the oracle's density matrix, n = 5 .. 13 (the paper's
3 .. 13; no 4-regular graph exists on 3 or 4 vertices).  The paper's fixed
angles come from a reference it does not reproduce, so one seeded angle set
stands in for them (the same for every n, as in the paper).  The fit of
Error = alpha exp(delta n - mu ln K) is printed (pytest -s) next to the paper's
alpha = 0.05737, delta = 0.11164, mu = 0.98682 (tests/golden/paper_numbers.json).

What is asserted, and against what:
  * the K law: Error ~ 1/K at every n (slope of log Error against log K) and mu;
  * the n law against the oracle's prediction for these circuits: Error has
    expectation (1/4K) sum_x Var_t(phi_x) / sigma_exact,x (delta method: Error is
    quadratic in sigma_approx - sigma_exact), with Var_t(phi_x) taken from the
    oracle's trajectories; the measured mean Error (K >= 100) must lie within
    [0.75, 1.33] of it at every n, and the fitted delta within 0.06 of the
    prediction's;
  * the fidelity band against the oracle's exact values for these circuits:
    the mean fidelity of sigma_approx to the uniform and to the noiseless
    distribution within 0.01 of the mean of F(sigma_exact, .) over n.
With substitute angles delta, alpha and the fidelity band are those of these
circuits, not the paper's numbers, which the test therefore does not assert.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
NS = (5, 6, 7, 8, 9, 10, 11, 12, 13)
KS = (10, 32, 100, 316, 1000, 1780)
SEEDS = 16


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


def predicted_error_numerator(n, edges, gates, G, noise, se, samples=20000, chunk=2000):
    """V_n = sum_x Var_t(phi_x) / (4 sigma_exact,x) from the oracle's trajectories, so
    that E[Error] ~ V_n / K (the delta method, Sec. "Results": Error ~ 1/K)."""
    s1 = np.zeros(1 << n)
    s2 = np.zeros(1 << n)
    nz = oracle.make_noise(**noise)
    for t0 in range(0, samples, chunk):
        phi = np.abs(oracle.traj_run(n, edges, gates, G, nz, 0x7A11E0 + n, t0, chunk, want_branches=False)["amps"]) ** 2
        s1 += phi.sum(axis=0)
        s2 += (phi ** 2).sum(axis=0)
    var = s2 / samples - (s1 / samples) ** 2
    return float(np.sum(var / (4.0 * se)))


def test_eq2_refit(qn):
    exp = GOLD["experiment"]
    noise = dict(p1=exp["lambda1"], p2=exp["lambda2"], damping=0.0, param=1)
    rows = []  # (n, K, mean Error, predicted Error)
    fid_uniform, fid_noiseless = [], []
    exact_uniform, exact_noiseless = [], []
    g, b = W.angles(exp["p"], 9100)  # one angle set for every n, as the paper fixes its angles
    for n in NS:
        edges = W.regular_graph(n, exp["degree"], 9000 + n)
        gates, G = oracle.qaoa_gates(n, edges, g, b)
        se = oracle.dm_run(n, edges, gates, G, oracle.make_noise(**noise))["diag"]
        ideal = np.abs(oracle.traj_run(n, edges, gates, G, oracle.make_noise(), 1, 0, 1)["amps"][0]) ** 2
        uniform = np.full(1 << n, 1.0 / (1 << n))
        exact_uniform.append(1 - oracle.error(se, uniform))
        exact_noiseless.append(1 - oracle.error(se, ideal))
        vn = predicted_error_numerator(n, edges, gates, G, noise, se)
        for K in KS:
            errs = []
            for s in range(SEEDS):
                with qn.Batch(n, K, 0x2210000000 + 1000 * n + 10 * s + KS.index(K)) as bt:
                    bt.run_qaoa(edges, g, b, **noise)
                    sa = bt.probs()
                errs.append(oracle.error(sa, se))
                fid_uniform.append(1 - oracle.error(sa, uniform))
                fid_noiseless.append(1 - oracle.error(sa, ideal))
            rows.append((n, K, float(np.mean(errs)), vn / K))
    n_arr = np.array([r[0] for r in rows], dtype=float)
    k_arr = np.array([r[1] for r in rows], dtype=float)
    e_arr = np.array([r[2] for r in rows])
    p_arr = np.array([r[3] for r in rows])
    A = np.stack([np.ones_like(n_arr), n_arr, -np.log(k_arr)], axis=1)

    def fit(e):
        y = np.log(e)
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        resid = y - A @ coef
        r2 = 1 - (resid ** 2).sum() / ((y - y.mean()) ** 2).sum()
        return float(np.exp(coef[0])), float(coef[1]), float(coef[2]), float(r2)

    alpha, delta, mu, r2 = fit(e_arr)
    p_alpha, p_delta, p_mu, p_r2 = fit(p_arr)
    paper = GOLD["eq2_error_model"]
    big = k_arr >= 100
    ratio = {int(n): float(np.mean(e_arr[big & (n_arr == n)] / p_arr[big & (n_arr == n)])) for n in NS}
    print(json.dumps({"fit": {"alpha": alpha, "delta": delta, "mu": mu, "r2": r2},
                      "oracle_prediction_fit": {"alpha": p_alpha, "delta": p_delta, "mu": p_mu},
                      "measured_over_predicted_K_ge_100": ratio,
                      "paper": {k: paper[k] for k in ("alpha", "delta", "mu", "r2")},
                      "mean_fidelity": {"to_uniform": float(np.mean(fid_uniform)),
                                        "to_noiseless": float(np.mean(fid_noiseless))},
                      "exact_fidelity": {"to_uniform": float(np.mean(exact_uniform)),
                                         "to_noiseless": float(np.mean(exact_noiseless))},
                      "paper_fidelity": GOLD["mean_fidelity"],
                      "grid": {"n": NS, "K": KS, "seeds_per_point": SEEDS}}))
    # Error ~ 1/K at every n (the slope of log Error against log K), and overall
    for n in NS:
        sel = n_arr == n
        slope = np.polyfit(np.log(k_arr[sel]), np.log(e_arr[sel]), 1)[0]
        assert 0.8 < -slope < 1.2, (n, slope)
    assert 0.85 < mu < 1.15, mu
    # the n law: the measured Error follows the oracle's prediction for these circuits (the
    # band covers the spread of a mean over 64 ensembles: repeated oracle-only runs of
    # this procedure gave ratios 0.87 .. 1.09)
    for n, r in ratio.items():
        assert 0.75 < r < 1.33, (n, r)
    assert abs(delta - p_delta) < 0.06, (delta, p_delta)
    # the fidelity band: sigma_approx's fidelities sit at sigma_exact's (minus O(1/K))
    assert abs(np.mean(fid_uniform) - np.mean(exact_uniform)) < 0.01
    assert abs(np.mean(fid_noiseless) - np.mean(exact_noiseless)) < 0.01

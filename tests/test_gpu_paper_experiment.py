"""The paper's experiment (Sec. "Results", Eq. 2) rerun on the GPU path.

QAOA p=2 on seeded 4-regular graphs, depolarizing noise with the paper's
lambda parameterisation (lambda1 = 1e-3 after 1q gates, lambda2 = 4e-3 after 2q
gates), ensembles of K = 10 .. 1780 circuits, Error = 1 - F(sigma_approx,
sigma_exact) against the oracle's density matrix.  The paper's fixed angles
come from a reference it does not reproduce, so one seeded angle set stands
in for them (the same for every n, as in the paper); the fit
of Error = alpha exp(delta n - mu ln K) is then compared with the paper's
structure: mu close to 1 (Error ~ 1/K) and delta > 0 (error grows with n).  With a substitute angle set the n dependence is not the paper's (delta and
alpha depend on the circuits), so only the K law is asserted: per n and overall.
The fitted numbers are printed (pytest -s) next to the paper's
alpha = 0.05737, delta = 0.11164, mu = 0.98682 (tests/golden/paper_numbers.json).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2210_15874_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))
NS = (5, 6, 7, 8, 9, 10, 11)
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


def test_eq2_refit(qn):
    exp = GOLD["experiment"]
    noise = dict(p1=exp["lambda1"], p2=exp["lambda2"], damping=0.0, param=1)
    rows = []  # (n, K, mean Error)
    fid_uniform, fid_noiseless = [], []
    g, b = W.angles(exp["p"], 9100)  # one angle set for every n, as the paper fixes its angles
    for n in NS:
        edges = W.regular_graph(n, exp["degree"], 9000 + n)
        gates, G = oracle.qaoa_gates(n, edges, g, b)
        se = oracle.dm_run(n, edges, gates, G, oracle.make_noise(**noise))["diag"]
        ideal = oracle.dm_run(n, edges, gates, G, oracle.make_noise())["diag"]
        uniform = np.full(1 << n, 1.0 / (1 << n))
        for K in KS:
            errs = []
            for s in range(SEEDS):
                with qn.Batch(n, K, 0x2210000000 + 1000 * n + 10 * s + KS.index(K)) as bt:
                    bt.run_qaoa(edges, g, b, **noise)
                    sa = bt.probs()
                errs.append(oracle.error(sa, se))
                fid_uniform.append(1 - oracle.error(sa, uniform))
                fid_noiseless.append(1 - oracle.error(sa, ideal))
            rows.append((n, K, float(np.mean(errs))))
    n_arr = np.array([r[0] for r in rows], dtype=float)
    k_arr = np.array([r[1] for r in rows], dtype=float)
    e_arr = np.array([r[2] for r in rows])
    A = np.stack([np.ones_like(n_arr), n_arr, -np.log(k_arr)], axis=1)
    y = np.log(e_arr)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    resid = y - A @ coef
    r2 = 1 - (resid ** 2).sum() / ((y - y.mean()) ** 2).sum()
    alpha, delta, mu = float(np.exp(coef[0])), float(coef[1]), float(coef[2])
    paper = GOLD["eq2_error_model"]
    print(json.dumps({"fit": {"alpha": alpha, "delta": delta, "mu": mu, "r2": r2},
                      "paper": {k: paper[k] for k in ("alpha", "delta", "mu", "r2")},
                      "mean_fidelity": {"to_uniform": float(np.mean(fid_uniform)),
                                        "to_noiseless": float(np.mean(fid_noiseless))},
                      "paper_fidelity": GOLD["mean_fidelity"],
                      "grid": {"n": NS, "K": KS, "seeds_per_point": SEEDS}}))
    # Error ~ 1/K at every n (the slope of log Error against log K), and overall
    for n in NS:
        sel = n_arr == n
        slope = np.polyfit(np.log(k_arr[sel]), y[sel], 1)[0]
        assert 0.8 < -slope < 1.2, (n, slope)
    assert 0.85 < mu < 1.15, mu
    assert delta > 0.0, delta  # error grows with the number of qubits
    assert 0.0 < np.mean(fid_uniform) <= 1.0 and 0.0 < np.mean(fid_noiseless) <= 1.0

"""Adjoint gradient (qn_grad, qn_grad_traj) against the FP64 oracle.

Per trajectory: central finite differences of the oracle's <C>_t with common
random numbers (the Philox draws do not depend on the angles, so the +-h runs
follow the same Kraus string), h = 1e-3.  Ensemble: the density-matrix gradient
(central differences of Tr(rho C), h = 1e-5) within 3 sigma/sqrt(K).
"""
import numpy as np
import pytest

import oracle
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


def fd_traj(w, t0, count, h=1e-3):
    """Central differences of the oracle's per-trajectory <C>_t in every angle."""
    nz = oracle.make_noise(**w.noise_kwargs())
    out = np.zeros((count, 2 * w.p))
    for k in range(2 * w.p):
        vals = []
        for sgn in (1, -1):
            g, b = w.gammas.copy(), w.betas.copy()
            (g if k % 2 == 0 else b)[k // 2] += sgn * h
            gates, G = oracle.qaoa_gates(w.n, w.edges, g, b)
            vals.append(oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, t0, count, want_amps=False,
                                        want_branches=False)["c_traj"])
        out[:, k] = (vals[0] - vals[1]) / (2 * h)
    return out[:, 0::2], out[:, 1::2]


def test_grad_traj_matches_crn_finite_differences(qn):
    w = W.qaoa_workload("grad_n10", 10, 2, index=21, trajectories=24, batch=24, p1=1e-2, p2=3e-2)
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=10) as b:
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        dg, db = b.grad_traj(0, w.trajectories)
    fg, fb = fd_traj(w, 0, w.trajectories)
    tol = 8 * U32 * w.gate_count * len(w.edges) + 1e-4
    assert np.abs(dg - fg).max() < tol, np.abs(dg - fg).max()
    assert np.abs(db - fb).max() < tol, np.abs(db - fb).max()
    assert np.abs(fg).max() > 0.1  # the case has non-trivial gradients


def test_grad_full_size_gradient_workload_sampled(qn):
    """16 qubits, p=6 (12 angles), K=2048 in one launch batch: the ensemble gradient runs
    at full size from the states the forward run left; sampled trajectories (re-simulated)
    are checked against the oracle, and the ensemble gradient equals the mean of the
    per-trajectory ones."""
    w = W.gradient_n16()
    with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        dg, db = b.grad()
        assert dg.shape == (6,) and db.shape == (6,) and np.all(np.isfinite(dg)) and np.all(np.isfinite(db))
        tg_all, tb_all = b.grad_traj(0, w.trajectories)  # re-simulates the whole ensemble
        np.testing.assert_allclose(tg_all.mean(axis=0), dg, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(tb_all.mean(axis=0), db, rtol=1e-9, atol=1e-12)
        for t in (0, 777, 2047):
            tg, tb = b.grad_traj(t, 1)
            fg, fb = fd_traj(w, t, 1)
            tol = 8 * U32 * w.gate_count * len(w.edges) + 1e-4
            assert np.abs(tg - fg).max() < tol and np.abs(tb - fb).max() < tol


def test_ensemble_grad_within_3_sigma_of_density_matrix(qn):
    w = W.qaoa_workload("grad_dm_n10", 10, 1, index=22, trajectories=1024, batch=256, p1=2e-2, p2=5e-2)
    with qn.Batch(w.n, w.trajectories, w.seed) as b:
        b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
        dg, db = b.grad()
        tg, tb = b.grad_traj(0, w.trajectories)
    np.testing.assert_allclose(dg, tg.mean(axis=0), rtol=1e-12, atol=1e-12)
    nz = oracle.make_noise(**w.noise_kwargs())
    h = 1e-5
    for k, (gpu_mean, per_traj) in enumerate([(dg[0], tg[:, 0]), (db[0], tb[:, 0])]):
        vals = []
        for sgn in (1, -1):
            g, bb = w.gammas.copy(), w.betas.copy()
            (g if k == 0 else bb)[0] += sgn * h
            gates, G = oracle.qaoa_gates(w.n, w.edges, g, bb)
            vals.append(oracle.dm_run(w.n, w.edges, gates, G, nz)["c"])
        exact = (vals[0] - vals[1]) / (2 * h)
        sigma = per_traj.std()
        assert abs(gpu_mean - exact) < 3 * sigma / np.sqrt(w.trajectories) + 1e-6, (k, gpu_mean, exact, sigma)


def test_grad_needs_pauli_only_noise(qn):
    with qn.Batch(4, 8, 3) as b:
        b.run_qaoa(W.ring_graph(4), [0.3], [0.2], p1=0.01, p2=0.01, damping=0.1)
        with pytest.raises(qn.QnError, match="QN_EINVAL"):
            b.grad()
    with qn.Batch(4, 8, 3) as b:
        b.run_qaoa(W.ring_graph(4), [], [], p1=0.01)
        dg, db = b.grad()
        assert dg.size == 0 and db.size == 0


def test_autograd_function_uses_the_adjoint(qn):
    import torch

    from paper_2210_15874_gb300.autograd import qaoa_energy

    w = W.qaoa_workload("grad_autograd_n8", 8, 2, index=23, trajectories=64, batch=64, p1=1e-2, p2=2e-2)
    g = torch.tensor(w.gammas, dtype=torch.float64, requires_grad=True)
    bt = torch.tensor(w.betas, dtype=torch.float64, requires_grad=True)
    with qn.Batch(w.n, w.trajectories, w.seed) as b:
        e = qaoa_energy(g, bt, b, w.edges, **w.noise_kwargs())
        (2.0 * e).backward()
        dg, db = b.grad()
    np.testing.assert_allclose(g.grad.numpy(), 2.0 * dg, rtol=1e-12)
    np.testing.assert_allclose(bt.grad.numpy(), 2.0 * db, rtol=1e-12)


def test_autograd_two_forwards_on_one_batch(qn):
    """Two energies at different angles on the same Batch summed into one loss: each
    backward must return the gradient at its own forward's angles, not at the angles
    the handle ran last."""
    import torch

    from paper_2210_15874_gb300.autograd import qaoa_energy

    w = W.qaoa_workload("grad_autograd_two", 8, 2, index=24, trajectories=64, batch=64, p1=1e-2, p2=2e-2)
    g1 = torch.tensor(w.gammas, dtype=torch.float64, requires_grad=True)
    b1 = torch.tensor(w.betas, dtype=torch.float64, requires_grad=True)
    g2 = torch.tensor(w.gammas[::-1].copy() + 0.3, dtype=torch.float64, requires_grad=True)
    b2 = torch.tensor(w.betas[::-1].copy() + 0.2, dtype=torch.float64, requires_grad=True)
    ref = []
    for g, bt in ((g1, b1), (g2, b2)):  # each on a fresh handle
        with qn.Batch(w.n, w.trajectories, w.seed) as b:
            b.run_qaoa(w.edges, g.detach().numpy(), bt.detach().numpy(), **w.noise_kwargs())
            ref.append(b.grad())
    assert np.abs(ref[0][0] - ref[1][0]).max() > 1e-3  # the two points differ
    with qn.Batch(w.n, w.trajectories, w.seed) as b:
        loss = qaoa_energy(g1, b1, b, w.edges, **w.noise_kwargs()) + 3.0 * qaoa_energy(
            g2, b2, b, w.edges, **w.noise_kwargs())
        loss.backward()
    np.testing.assert_allclose(g1.grad.numpy(), ref[0][0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b1.grad.numpy(), ref[0][1], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g2.grad.numpy(), 3.0 * ref[1][0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b2.grad.numpy(), 3.0 * ref[1][1], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n,p,d", [(2, 2, 1), (3, 2, 2), (5, 2, 4), (8, 3, 3), (9, 2, 4), (11, 2, 4), (12, 2, 3),
                                   (13, 2, 4), (14, 2, 3), (15, 2, 4), (16, 2, 3), (17, 1, 4)])
def test_fused_adjoint_matches_per_gate_adjoint_and_oracle(qn, n, p, d):
    """The fused adjoint (what the default fused mode runs) against the one reverse sweep
    per gate (fusion off) on the same trajectories, and against CRN finite differences of
    the oracle.  Below 12 qubits the reverse takes a layer's mixer in register windows of
    two to four qubits and its cost diagonal in a sweep of its own: the qubit-0 window
    alone (n = 2, 3), a single-qubit window (n = 5), windows of two and three (n = 8-11).
    From 12 on it takes tiles through shared memory: qubits 0-9, then windows of two to
    six qubits, the last with the cost diagonal (n = 12-16: one window of 2-6; n = 17:
    4 + 3)."""
    if n == 2:  # the one-edge graph
        w = W.Workload("fadj_n2", 2, np.array([[0, 1]], np.int32), p, *W.angles(p, 4462), 1e-2, 3e-2, 0.0, 32, 32,
                       W.PHILOX_SEED_BASE + 42)
    else:
        w = W.qaoa_workload(f"fadj_n{n}", n, p, index=40 + n, trajectories=32, batch=32, p1=1e-2, p2=3e-2, d=d)
    res = {}
    for fusion in (True, False):
        with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
            b.set_fusion(fusion)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            res[fusion] = b.grad_traj(0, w.trajectories)
    tol = 8 * U32 * w.gate_count * len(w.edges) + 1e-4
    for k in range(2):
        assert np.abs(res[True][k] - res[False][k]).max() < tol, (k, np.abs(res[True][k] - res[False][k]).max())
    fg, fb = fd_traj(w, 0, 8)
    assert np.abs(res[True][0][:8] - fg).max() < tol
    assert np.abs(res[True][1][:8] - fb).max() < tol
    assert np.abs(fg).max() + np.abs(fb).max() > 0.05  # non-trivial gradients


def test_tiled_adjoint_two_windows_n20(qn):
    """n = 20 (qubits 0-9, then two windows of five: a plain one and the one with the
    cost diagonal), 64 trajectories over two launch batches: the fused adjoint against
    the one reverse sweep per gate on the same trajectories."""
    w = W.qaoa_workload("fadj_n20", 20, 2, index=60, trajectories=64, batch=32, p1=1e-2, p2=3e-2)
    res = {}
    for fusion in (True, False):
        with qn.Batch(w.n, w.trajectories, w.seed, launch_batch=w.batch) as b:
            b.set_fusion(fusion)
            b.run_qaoa(w.edges, w.gammas, w.betas, **w.noise_kwargs())
            res[fusion] = b.grad_traj(0, w.trajectories)
    tol = 8 * U32 * w.gate_count * len(w.edges) + 1e-4
    for k in range(2):
        assert np.abs(res[True][k] - res[False][k]).max() < tol, (k, np.abs(res[True][k] - res[False][k]).max())
    assert np.abs(res[False][0]).max() + np.abs(res[False][1]).max() > 0.05

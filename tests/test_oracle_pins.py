"""Pins of the FP64 CPU oracle against facts fixed outside it.

Each test names what it pins.  None of them re-types an oracle formula: they use
closed forms (Pauli twirl, Wang et al. p=1 QAOA, damping decay), brute-force
enumeration of Kraus strings, an independent library (cuRAND's host Philox),
and statistics.
"""
import ctypes
import ctypes.util
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2210_15874_gb300 import workloads

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def random_rho(n, rng):
    d = 1 << n
    a = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    r = a @ a.conj().T
    return np.ascontiguousarray(r / np.trace(r))


def bloch(rho):
    return np.real([np.trace(rho @ P) for P in (X, Y, Z)])


# --------------------------------------------------------------------------- Philox
def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_philox_matches_curand_host_generator():
    """P9: the oracle's Philox4x32-10 equals cuRAND's host PHILOX4_32_10 generator.

    cuRAND's host generator with seed s produces, for output block j, Philox4x32-10
    at counter (0, 0, j, 0) with key (s_lo, s_hi) for j < 2^16; the generator
    offset (4 j) selects the block.  Checked on several seeds and block ranges."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not found")
    for seed in (0, 1, 0x2210158740000001, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF):
        for first_block in (0, 7, 1000, 65530):
            gen = ctypes.c_void_p()
            assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            assert cr.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
            nblk = 6
            out = np.zeros(4 * nblk, dtype=np.uint32)
            assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
            cr.curandDestroyGenerator(gen)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for b in range(nblk):
                j = first_block + b
                mine = oracle.philox4x32_10([0, 0, j & 0xFFFFFFFF, j >> 32], key)
                assert list(mine) == list(out[4 * b:4 * b + 4]), (seed, j)


def test_philox_counter_words_distinct_streams():
    """Every counter word and key word changes the output (no ignored input)."""
    base = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] ^= 1
        assert list(oracle.philox4x32_10(c, [5, 6])) != list(base)
    for k in range(2):
        kk = [5, 6]
        kk[k] ^= 1
        assert list(oracle.philox4x32_10([1, 2, 3, 4], kk)) != list(base)


# --------------------------------------------------------------------------- channels
@pytest.mark.parametrize("p", [0.0, 1e-3, 0.2, 0.75])
def test_depolarizing_1q_bloch_shrink(p):
    """P1: the 1q depolarizing channel shrinks the Bloch vector by 1 - 4p/3
    (= 1 - lambda with the paper's Kraus set, Sec. "Modeling Noise")."""
    rng = np.random.default_rng(1)
    rho = random_rho(1, rng)
    b0 = bloch(rho)
    oracle.dm_depolarize_1q(rho, 1, 0, oracle.make_noise(p1=p))
    np.testing.assert_allclose(bloch(rho), (1 - 4 * p / 3) * b0, atol=1e-14)
    assert abs(np.trace(rho) - 1) < 1e-14
    lam = 4 * p / 3
    rho2 = random_rho(1, rng)
    b2 = bloch(rho2)
    oracle.dm_depolarize_1q(rho2, 1, 0, oracle.make_noise(p1=lam, param=1))
    np.testing.assert_allclose(bloch(rho2), (1 - lam) * b2, atol=1e-14)


def _ptrace_keep(rho, n, keep):
    """Reduced density matrix on the qubits in `keep` (in that order)."""
    t = rho.reshape([2] * (2 * n))
    # axis a (a < n) is bit n-1-a of the row index; axis n+a the same for columns
    ax = lambda q: n - 1 - q
    others = [q for q in range(n) if q not in keep]
    letters = "abcdefghijklmnopqrstuvwxyz"
    rows = [letters[i] for i in range(n)]
    cols = [letters[n + i] for i in range(n)]
    for q in others:
        cols[ax(q)] = rows[ax(q)]
    out = "".join(rows[ax(q)] for q in keep) + "".join(cols[ax(q)] for q in keep)
    r = np.einsum("".join(rows) + "".join(cols) + "->" + out, t)
    d = 1 << len(keep)
    # row index of r: first kept qubit is the most significant of the reshaped axes
    return r.reshape(d, d)


def _embed_identity(rho_rest, n, q0, q1):
    """(Tr_{q0 q1} rho) (x) I/4 placed back on qubits q0, q1."""
    d = 1 << n
    out = np.zeros((d, d), dtype=np.complex128)
    rest = [q for q in range(n) if q not in (q0, q1)]
    for r in range(d):
        for c in range(d):
            if ((r >> q0) & 1) != ((c >> q0) & 1) or ((r >> q1) & 1) != ((c >> q1) & 1):
                continue
            rr = sum(((r >> q) & 1) << (len(rest) - 1 - k) for k, q in enumerate(rest))
            cc = sum(((c >> q) & 1) << (len(rest) - 1 - k) for k, q in enumerate(rest))
            out[r, c] = rho_rest[rr, cc] / 4
    return out


@pytest.mark.parametrize("p", [1e-2, 0.3, 15 / 16])
def test_depolarizing_2q_pauli_twirl(p):
    """2q depolarizing with each non-II Pauli at p/15 equals
    (1 - 16p/15) rho + (16p/15) Tr_ij(rho) (x) I/4 (Pauli-twirl identity).
    At p = 15/16 the pair is left fully mixed."""
    n, q0, q1 = 3, 2, 0
    rng = np.random.default_rng(2)
    rho = random_rho(n, rng)
    ref = rho.copy()
    oracle.dm_depolarize_2q(rho, n, q0, q1, oracle.make_noise(p2=p))
    rest = _ptrace_keep(ref, n, [1])
    expect = (1 - 16 * p / 15) * ref + (16 * p / 15) * _embed_identity(rest, n, q0, q1)
    np.testing.assert_allclose(rho, expect, atol=1e-14)
    # paper's lambda: K0 weight 1 - 15 lambda / 16
    rho2 = ref.copy()
    oracle.dm_depolarize_2q(rho2, n, q0, q1, oracle.make_noise(p2=16 * p / 15, param=1))
    np.testing.assert_allclose(rho2, expect, atol=1e-14)


def test_depolarizing_2q_product_mode_is_two_1q_channels():
    """twoq_mode=1 (Fig. 2 semantics) equals the 1q closed form applied to each qubit."""
    n, p = 2, 0.2
    rng = np.random.default_rng(3)
    rho = random_rho(n, rng)
    ref = rho.copy()
    oracle.dm_depolarize_2q(rho, n, 0, 1, oracle.make_noise(p2=p, twoq_mode=1))
    # closed form of a 1q depolarizing on qubit q: (1 - 4p/3) rho + (4p/3) Tr_q(rho) (x) I/2
    def dep1(r, q):
        d = 1 << n
        out = (1 - 4 * p / 3) * r
        bit = 1 << q
        for a in range(d):
            for c in range(d):
                if (a & bit) != (c & bit):
                    continue
                tr = r[a & ~bit, c & ~bit] + r[a | bit, c | bit]
                out[a, c] += (4 * p / 3) * tr / 2
        return out
    np.testing.assert_allclose(rho, dep1(dep1(ref, 0), 1), atol=1e-14)


def test_fig2_product_probabilities():
    """Fig. 2: per-qubit noise on a 2q gate gives no noise (1-p)^2, one qubit p(1-p)
    each, both p^2 -- in the oracle's table and in sampled Kraus strings."""
    p = 0.3
    nz = oracle.make_noise(p1=0.0, p2=p, twoq_mode=1)
    pr = oracle.pauli_probs(nz, True).reshape(4, 4)
    assert abs(pr[0, 0] - (1 - p) ** 2) < 1e-15
    assert abs(pr[0, 1:].sum() - p * (1 - p)) < 1e-15
    assert abs(pr[1:, 0].sum() - p * (1 - p)) < 1e-15
    assert abs(pr[1:, 1:].sum() - p * p) < 1e-15
    # sampled: n=2 single edge, p=1 circuit; count 2q codes over trajectories
    edges = np.array([[0, 1]], dtype=np.int32)
    gates, G = oracle.qaoa_gates(2, edges, [0.3], [0.2])
    K = 40000
    r = oracle.traj_run(2, edges, gates, G, nz, 77, 0, K, want_amps=False)
    codes = r["branches"][:, 2] & 15
    a, b = codes >> 2, codes & 3
    for frac, expect in (((a == 0) & (b == 0), (1 - p) ** 2), ((a != 0) & (b != 0), p * p),
                         ((a != 0) & (b == 0), p * (1 - p))):
        f = frac.mean()
        assert abs(f - expect) < 5 * np.sqrt(expect * (1 - expect) / K)


def test_thresholds_edges():
    """T_k = floor(2^32 c_k); p = 0 puts every word in bucket 0."""
    t = oracle.thresholds([1.0, 0.0, 0.0, 0.0])
    assert t[0] == 1 << 32
    t = oracle.thresholds([0.5, 0.25, 0.125, 0.125])
    assert list(t) == [1 << 31, 3 << 30, 7 << 29, 1 << 32]


@pytest.mark.parametrize("gamma", [0.05, 0.5, 1.0])
def test_damping_closed_forms(gamma):
    """P5: |1> after m damping sites keeps P(1) = (1-gamma)^m; the |+> coherence
    is multiplied by sqrt(1-gamma) per site."""
    rho = np.zeros((2, 2), dtype=np.complex128)
    rho[1, 1] = 1
    plus = np.full((2, 2), 0.5, dtype=np.complex128)
    for m in range(1, 5):
        oracle.dm_damp(rho, 1, 0, gamma)
        oracle.dm_damp(plus, 1, 0, gamma)
        assert abs(rho[1, 1].real - (1 - gamma) ** m) < 1e-14
        assert abs(rho[0, 0].real - (1 - (1 - gamma) ** m)) < 1e-14
        assert abs(plus[0, 1] - 0.5 * (1 - gamma) ** (m / 2)) < 1e-14


def test_dm_physical_after_every_channel():
    """P3: rho stays Hermitian with unit trace and nonnegative spectrum after
    every gate and every channel."""
    n = 4
    edges = workloads.ring_graph(n)
    nz = oracle.make_noise(p1=0.05, p2=0.1, damping=0.1)
    gates, G = oracle.qaoa_gates(n, edges, [0.7, 1.9], [0.4, 2.5])
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1
    for g in range(G):
        gt = gates[g]
        oracle.dm_gate(rho, n, gt.kind, gt.q0, gt.q1, gt.angle)
        steps = []
        if gt.kind == oracle.ZZ:
            steps.append(lambda: oracle.dm_depolarize_2q(rho, n, gt.q0, gt.q1, nz))
            steps.append(lambda: oracle.dm_damp(rho, n, gt.q0, nz.damping))
            steps.append(lambda: oracle.dm_damp(rho, n, gt.q1, nz.damping))
        else:
            steps.append(lambda: oracle.dm_depolarize_1q(rho, n, gt.q0, nz))
            steps.append(lambda: oracle.dm_damp(rho, n, gt.q0, nz.damping))
        for s in steps:
            s()
            assert np.abs(rho - rho.conj().T).max() < 1e-14
            assert abs(np.trace(rho) - 1) < 1e-13
            assert np.linalg.eigvalsh(rho).min() > -1e-12
    full = oracle.dm_run(n, edges, gates, G, nz, want_rho=True)["rho"]
    np.testing.assert_allclose(full, rho, atol=1e-13)


# --------------------------------------------------------------------------- QAOA closed form
def wang_p1_edge(gamma, beta, du, dv, lam):
    """<C_uv> for p=1 QAOA (Wang, Hadfield, Jiang, Rieffel, PRA 97, 022304 (2018)),
    du, dv = degrees, lam = common neighbours, C_uv = (1 - Z_u Z_v)/2."""
    c = np.cos(gamma)
    return (0.5 + 0.25 * np.sin(4 * beta) * np.sin(gamma) * (c ** (du - 1) + c ** (dv - 1))
            - 0.25 * np.sin(2 * beta) ** 2 * c ** (du + dv - 2 - 2 * lam) * (1 - np.cos(2 * gamma) ** lam))


def wang_p1(n, edges, gamma, beta):
    adj = [set() for _ in range(n)]
    for i, j in edges:
        adj[i].add(j)
        adj[j].add(i)
    return sum(wang_p1_edge(gamma, beta, len(adj[i]), len(adj[j]), len(adj[i] & adj[j])) for i, j in edges)


@pytest.mark.parametrize("graph", ["ring6", "ring8", "reg3_n8", "reg3_n10"])
def test_noiseless_p1_closed_form(graph):
    """P2: noiseless p=1 <C> of O1 and O2 equals the analytic formula (fixes the
    circuit conventions: ZZ phase, RX sign, gate order, bit order)."""
    if graph.startswith("ring"):
        n = int(graph[4:])
        edges = workloads.ring_graph(n)
    else:
        n = int(graph.split("n")[-1])
        edges = workloads.regular_graph(n, 3, 11 + n)
    nz = oracle.make_noise()
    for gamma, beta in ((0.3, 0.7), (1.1, 2.6), (2.9, 0.15)):
        expect = wang_p1(n, edges, gamma, beta)
        gates, G = oracle.qaoa_gates(n, edges, [gamma], [beta])
        dm = oracle.dm_run(n, edges, gates, G, nz)
        tr = oracle.traj_run(n, edges, gates, G, nz, 5, 0, 1)
        assert abs(dm["c"] - expect) < 1e-12
        assert abs(tr["c_traj"][0] - expect) < 1e-12
        if graph.startswith("ring"):
            assert abs(expect - n * (0.5 + 0.25 * np.sin(4 * beta) * np.sin(2 * gamma))) < 1e-12


@pytest.mark.parametrize("graph", ["ring7", "reg3_n8", "reg3_n10"])
def test_noiseless_multilayer_reduces_to_p1_closed_form(graph):
    """P2 for p >= 2, pinning the oracle's layer loop (which angle goes to which
    layer, and the order of the cost and mixer halves within a layer).

    A layer with beta = 0 has the identity mixer, and U_C(gamma) commutes with
    C and with every other U_C.  So, noiseless:
      (gamma1, 0), (gamma2, beta2)              -> Wang p=1 at (gamma1 + gamma2, beta2)
      (gamma2, beta2), (gamma1, 0)              -> Wang p=1 at (gamma2, beta2)
      (gamma1, 0), (gamma2, 0), (gamma3, beta3) -> Wang p=1 at (gamma1 + gamma2 + gamma3, beta3)
    A loop that reused layer 0's angles, swapped gamma and beta, or ran the mixer
    before the cost layer gives other values (checked to differ by > 1e-3 here)."""
    if graph.startswith("ring"):
        n = int(graph[4:])
        edges = workloads.ring_graph(n)
    else:
        n = int(graph.split("n")[-1])
        edges = workloads.regular_graph(n, 3, 29 + n)
    nz = oracle.make_noise()
    g1, g2, g3, b2, b3 = 0.37, 1.21, 0.58, 2.47, 0.83
    cases = [([g1, g2], [0.0, b2], wang_p1(n, edges, g1 + g2, b2)),
             ([g2, g1], [b2, 0.0], wang_p1(n, edges, g2, b2)),
             ([g1, g2, g3], [0.0, 0.0, b3], wang_p1(n, edges, g1 + g2 + g3, b3))]
    # the plausible layer-loop mistakes land elsewhere
    assert abs(cases[0][2] - wang_p1(n, edges, 2 * g1, b2)) > 1e-3      # gammas[0] reused
    assert abs(cases[0][2] - wang_p1(n, edges, g2, b2)) > 1e-3          # first layer dropped
    assert abs(cases[0][2] - cases[1][2]) > 1e-3                        # layers swapped
    for gammas, betas, expect in cases:
        gates, G = oracle.qaoa_gates(n, edges, gammas, betas)
        assert G == n + len(gammas) * (len(edges) + n)
        dm = oracle.dm_run(n, edges, gates, G, nz)
        tr = oracle.traj_run(n, edges, gates, G, nz, 5, 0, 1)
        assert abs(dm["c"] - expect) < 1e-12, (gammas, betas)
        assert abs(tr["c_traj"][0] - expect) < 1e-12, (gammas, betas)


def test_noiseless_dm_is_pure_trajectory():
    """P6: with p = gamma = 0, rho = |psi><psi| for the (single, deterministic) trajectory."""
    n = 5
    edges = workloads.ring_graph(n)
    gates, G = oracle.qaoa_gates(n, edges, [0.4, 1.3], [2.2, 0.9])
    nz = oracle.make_noise()
    rho = oracle.dm_run(n, edges, gates, G, nz, want_rho=True)["rho"]
    psi = oracle.traj_run(n, edges, gates, G, nz, 9, 3, 1)["amps"][0]
    np.testing.assert_allclose(rho, np.outer(psi, psi.conj()), atol=1e-13)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_full_depolarizing_leaves_last_qubit_mixed():
    """P6: p1 = 3/4 (fully depolarizing 1q channel) leaves the last-gated qubit in I/2."""
    n = 4
    edges = workloads.ring_graph(n)
    gates, G = oracle.qaoa_gates(n, edges, [0.8], [0.3])
    nz = oracle.make_noise(p1=0.75, p2=0.01)
    rho = oracle.dm_run(n, edges, gates, G, nz, want_rho=True)["rho"]
    last = gates[G - 1].q0
    red = _ptrace_keep(rho, n, [last])
    np.testing.assert_allclose(red, np.eye(2) / 2, atol=1e-14)


# --------------------------------------------------------------------------- unravelling
def _branch_space(gates, G, with_pauli, with_damp):
    per_gate = []
    for g in range(G):
        twoq = gates[g].kind == oracle.ZZ
        codes = range(16 if twoq else 4) if with_pauli else [0]
        jumps = range(4 if twoq else 2) if with_damp else [0]
        per_gate.append([c | (j << 4) for c in codes for j in jumps])
    return per_gate


@pytest.mark.parametrize("case", ["n1_both", "n2_pauli", "n2_damp", "n2_both"])
def test_bruteforce_unravelling_equals_dm(case):
    """P4: enumerating every Kraus string with its Born weight reproduces the
    density matrix: sum_w w |psi_w><psi_w| = rho, sum_w w = 1 (includes damping,
    pins the per-gate order gate -> Pauli -> damping(i) -> damping(j))."""
    n = int(case[1])
    with_pauli = case.endswith("pauli") or case.endswith("both")
    with_damp = case.endswith("damp") or case.endswith("both")
    edges = np.array([[0, 1]], dtype=np.int32) if n == 2 else np.zeros((0, 2), dtype=np.int32)
    nz = oracle.make_noise(p1=0.08 if with_pauli else 0.0, p2=0.12 if with_pauli else 0.0,
                           damping=0.3 if with_damp else 0.0)
    gates, G = oracle.qaoa_gates(n, edges, [0.9], [0.35])
    rho = oracle.dm_run(n, edges, gates, G, nz, want_rho=True)["rho"]
    acc = np.zeros_like(rho)
    wsum = 0.0
    for combo in itertools.product(*_branch_space(gates, G, with_pauli, with_damp)):
        psi, w = oracle.traj_forced(n, gates, G, nz, np.array(combo, dtype=np.uint8))
        if psi is None or w == 0.0:
            continue
        acc += w * np.outer(psi, psi.conj())
        wsum += w
    assert abs(wsum - 1) < 1e-12
    np.testing.assert_allclose(acc, rho, atol=1e-12)


def test_pauli_frame_identity():
    """P7: an X error right after H on qubit q equals the ideal circuit with the
    sign of gamma flipped on every edge at q followed by a final X_q; a Z error
    there equals flipping beta on every later RX of q followed by a final Z_q
    (up to a global phase)."""
    n = 4
    edges = workloads.ring_graph(n)
    gam, bet = [0.7, 1.6], [0.3, 2.1]
    gates, G = oracle.qaoa_gates(n, edges, gam, bet)
    nz = oracle.make_noise(p1=0.1, p2=0.1)
    q = 2
    for code, flip in ((1, "gamma"), (3, "beta")):
        forced = np.zeros(G, dtype=np.uint8)
        forced[q] = code
        psi_err, _ = oracle.traj_forced(n, gates, G, nz, forced)
        mod = []
        for g in range(G):
            gt = gates[g]
            ang = gt.angle
            if flip == "gamma" and gt.kind == oracle.ZZ and q in (gt.q0, gt.q1):
                ang = -ang
            if flip == "beta" and gt.kind == oracle.RX and gt.q0 == q:
                ang = -ang
            mod.append((gt.kind, gt.q0, gt.q1, ang))
        arr, Gm = oracle.gate_array(mod)
        psi_id, _ = oracle.traj_forced(n, arr, Gm, oracle.make_noise(), np.zeros(Gm, dtype=np.uint8))
        x = np.arange(1 << n)
        if code == 1:
            psi_id = psi_id[x ^ (1 << q)]
        else:
            psi_id = psi_id * np.where((x >> q) & 1, -1.0, 1.0)
        assert abs(abs(np.vdot(psi_id, psi_err)) - 1) < 1e-12


# --------------------------------------------------------------------------- statistics
@pytest.mark.slow
def test_ensemble_mean_within_3_sigma_of_dm():
    """P8(i): S1/K of O2 lies within 3 sigma/sqrt(K) of Tr(rho C) from O1 (20 seeds,
    allowing the ~0.5 expected 3-sigma excursions plus slack)."""
    n = 6
    edges = workloads.regular_graph(n, 3, 5)
    gates, G = oracle.qaoa_gates(n, edges, [0.6, 1.2], [0.9, 0.4])
    nz = oracle.make_noise(p1=0.02, p2=0.05, damping=0.05)
    exact = oracle.dm_run(n, edges, gates, G, nz)["c"]
    K = 512
    fails = 0
    for s in range(20):
        r = oracle.traj_run(n, edges, gates, G, nz, 1000 + s, 0, K, want_amps=False, want_branches=False)
        mean = r["s1"] / K
        var = r["s2"] / K - mean ** 2
        if abs(mean - exact) > 3 * np.sqrt(var / K):
            fails += 1
    assert fails <= 2


@pytest.mark.slow
def test_error_scales_as_one_over_K():
    """P8(ii): E[Error] = (1/4K) sum_x Var_t(phi_x) / sigma_exact_x (delta method),
    which makes Error * K flat in K -- the paper's Error ~ 1/K observation."""
    n = 5
    edges = workloads.ring_graph(n)
    gates, G = oracle.qaoa_gates(n, edges, [0.5, 1.1], [0.7, 0.2])
    nz = oracle.make_noise(p1=0.03, p2=0.06)
    se = oracle.dm_run(n, edges, gates, G, nz)["diag"]
    big = oracle.traj_run(n, edges, gates, G, nz, 99, 0, 20000, want_branches=False)
    phi = np.abs(big["amps"]) ** 2
    predicted_times_k = (phi.var(axis=0) / se).sum() / 4
    for K in (64, 256, 1024):
        errs = []
        for s in range(40):
            r = oracle.traj_run(n, edges, gates, G, nz, 5000 + 97 * s + K, 0, K, want_amps=False,
                                want_branches=False)
            errs.append(oracle.error(r["probs_sum"] / K, se))
        assert abs(np.mean(errs) * K / predicted_times_k - 1) < 0.25, K


# --------------------------------------------------------------------------- metric
def test_error_metric():
    """Eq. 1: Error(s, s) = 0, symmetric, in [0, 1]; two-outcome example 1/2."""
    rng = np.random.default_rng(4)
    s = rng.random(16)
    s /= s.sum()
    t = rng.random(16)
    t /= t.sum()
    assert abs(oracle.error(s, s)) < 1e-15
    assert abs(oracle.error(s, t) - oracle.error(t, s)) < 1e-15
    assert 0 <= oracle.error(s, t) <= 1
    assert abs(oracle.error([0.5, 0.5], [1.0, 0.0]) - 0.5) < 1e-15
    assert abs(oracle.error([0.0, 1.0], [1.0, 0.0]) - 1.0) < 1e-15

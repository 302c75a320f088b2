"""Seeded synthetic inputs: random regular graphs and QAOA angles.

This module holds input generation only -- none of the method's arithmetic.
It is the one module that both the CUDA path's callers and the CPU oracle's
tests draw their inputs from, so both sides always see the same graph, angles,
noise parameters and Philox seed.

The paper's workloads are QAOA MaxCut circuits on random regular graphs
(Sec. "Results": p = 2, d = 4, n = 3..13, fixed angles).  The fixed angles come
from a reference the paper does not reproduce, so angles are drawn here as
gamma, beta ~ U[0, pi) from a seeded numpy generator.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def regular_graph(n: int, d: int, seed: int, max_tries: int = 100000) -> np.ndarray:
    """Random simple d-regular graph on n vertices by the pairing (configuration)
    model with rejection of self-loops and multi-edges.

    Returns an int32 array [E, 2] with i < j in every row, rows sorted; E = n*d/2.
    The row order is the order in which the circuit applies the ZZ gates.
    """
    if n * d % 2 != 0 or d >= n:
        raise ValueError(f"no simple {d}-regular graph on {n} vertices")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        pairs = perm.reshape(-1, 2)
        a = np.minimum(pairs[:, 0], pairs[:, 1])
        b = np.maximum(pairs[:, 0], pairs[:, 1])
        if np.any(a == b):
            continue
        keys = a * n + b
        if len(np.unique(keys)) != len(keys):
            continue
        order = np.argsort(keys)
        return np.stack([a[order], b[order]], axis=1).astype(np.int32)
    raise RuntimeError("pairing model did not produce a simple graph")


def ring_graph(n: int) -> np.ndarray:
    """Cycle 0-1-...-(n-1)-0 as an int32 [n, 2] edge list (i < j per row)."""
    e = [(i, (i + 1) % n) for i in range(n)]
    return np.array([(min(a, b), max(a, b)) for a, b in e], dtype=np.int32)


def angles(p: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """gamma_l, beta_l ~ U[0, pi), l = 1..p, from a seeded generator."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.0, np.pi, size=p)
    b = rng.uniform(0.0, np.pi, size=p)
    return g.astype(np.float64), b.astype(np.float64)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named synthetic workload: graph, depth, angles, noise, ensemble size."""
    name: str
    n: int
    edges: np.ndarray
    p: int
    gammas: np.ndarray
    betas: np.ndarray
    p1: float
    p2: float
    damping: float
    trajectories: int
    batch: int
    seed: int
    twoq_mode: int = 0
    param: int = 0

    @property
    def gate_count(self) -> int:
        return self.n + self.p * (len(self.edges) + self.n)

    def noise_kwargs(self) -> dict:
        return dict(p1=self.p1, p2=self.p2, damping=self.damping, twoq_mode=self.twoq_mode,
                    param=self.param)


PHILOX_SEED_BASE = 0x2210158740000000


def qaoa_workload(name: str, n: int, p: int, *, index: int, trajectories: int, batch: int,
                  p1: float = 1e-3, p2: float = 1e-2, damping: float = 0.0, d: int = 3,
                  twoq_mode: int = 0, param: int = 0) -> Workload:
    """Seeded d-regular QAOA workload; graph seed 2210 + index, angle seed 4420 + index,
    Philox seed PHILOX_SEED_BASE + index."""
    edges = regular_graph(n, d, 2210 + index) if n > d else ring_graph(n)
    g, b = angles(p, 4420 + index)
    return Workload(name, n, edges, p, g, b, p1, p2, damping, trajectories, batch,
                    PHILOX_SEED_BASE + index, twoq_mode, param)


def plain_n8() -> Workload:
    """QAOA p=1 on a seeded 3-regular n=8 graph, depolarizing p1=1e-3 / p2=1e-2, K=1024."""
    return qaoa_workload("qaoa_n8_p1_depol_K1024", 8, 1, index=0, trajectories=1024, batch=1024)


def damping_n20() -> Workload:
    """QAOA p=3 on a seeded 3-regular n=20 graph, depolarizing plus amplitude damping
    gamma=5e-3 after every gate, K=4096, 64 statevectors per launch."""
    return qaoa_workload("qaoa_n20_p3_depol_damp_K4096", 20, 3, index=1, trajectories=4096, batch=64,
                         damping=5e-3)


def precision_n26() -> Workload:
    """QAOA p=4 on a seeded 3-regular n=26 graph, depolarizing only."""
    return qaoa_workload("qaoa_n26_p4_depol", 26, 4, index=2, trajectories=64, batch=64)


def precision_n30() -> Workload:
    """QAOA p=4 on a seeded 3-regular n=30 graph, depolarizing only, 16 trajectories
    of 8 GiB each in one launch."""
    return qaoa_workload("qaoa_n30_p4_depol", 30, 4, index=2, trajectories=16, batch=16)


def gradient_n16() -> Workload:
    """QAOA p=6 on a seeded 3-regular n=16 graph, depolarizing only, K=2048 in one launch
    batch (2048 states of 512 KiB, 1 GiB)."""
    return qaoa_workload("qaoa_n16_p6_depol_K2048", 16, 6, index=4, trajectories=2048, batch=2048)

"""Trajectory sharding of one ensemble over several ranks (one GPU each).

Trajectories are independent (the paper's sample parallelism, Sec.
"Parallelism Hierarchy"), and the library keys every random draw by the global
trajectory id (qn_batch_set_offset), so a contiguous id range per rank gives
each rank exactly the trajectories a single-GPU run would simulate.  The only
exchange is one sum of (S1, S2, sum |psi|^2) at the end -- host-side
arithmetic on the ranks' results, no collective on the data path.
"""
from __future__ import annotations

import numpy as np


def shard_range(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [first, first + count) of `total` trajectories for `rank`;
    the first total % world ranks take one extra."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def local_sums(mean: float, std_err: float, probs: np.ndarray, count: int) -> np.ndarray:
    """(S1, S2, sum_t |psi_t|^2) of one shard from qn_expectation / qn_probs outputs."""
    s1 = mean * count
    var = std_err * std_err * count
    s2 = (var + mean * mean) * count
    return np.concatenate([[s1, s2, float(count)], np.asarray(probs, dtype=np.float64) * count])


def finish(sums: np.ndarray) -> tuple[float, float, np.ndarray]:
    """Ensemble mean, standard error and sigma_approx from summed shard sums."""
    s1, s2, k = sums[0], sums[1], sums[2]
    mean = s1 / k
    var = max(0.0, s2 / k - mean * mean)
    return float(mean), float(np.sqrt(var / k)), sums[3:] / k


def allreduce_ensemble(mean, std_err, probs, count, group=None):
    """Sum the shards' (S1, S2, K, sigma sums) over the process group; returns the
    ensemble (mean, std_err, sigma_approx) on every rank."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(local_sums(mean, std_err, probs, count))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return finish(t.numpy())

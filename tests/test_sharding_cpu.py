"""Sharding an ensemble over ranks: world size 2 on CPU (gloo).

Each rank runs its contiguous trajectory range with the oracle (standing in for
the per-rank GPU run, which draws the same Philox words for the same global
ids) and the shards are combined with one all-reduce of the sums.  The result
must equal the single-process run of the whole ensemble."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2210_15874_gb300 import shards


def test_shard_ranges_partition():
    for total in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            got = [shards.shard_range(total, world, r) for r in range(world)]
            assert sum(c for _, c in got) == total
            pos = 0
            for first, count in got:
                assert first == pos
                pos += count
    with pytest.raises(ValueError):
        shards.shard_range(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import oracle
    from paper_2210_15874_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.qaoa_workload("shard_n6", 6, 2, index=11, trajectories=50, batch=50, p1=0.02, p2=0.05, damping=0.05)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    nz = oracle.make_noise(**w.noise_kwargs())
    first, count = shards.shard_range(w.trajectories, world, rank)
    r = oracle.traj_run(w.n, w.edges, gates, G, nz, w.seed, first, count, want_amps=False, threads=1)
    mean = r["s1"] / count
    se = np.sqrt(max(0.0, r["s2"] / count - mean * mean) / count)
    m, s, probs = shards.allreduce_ensemble(mean, se, r["probs_sum"] / count, count)
    out[rank] = (m, s, probs.tolist())
    dist.destroy_process_group()


def test_two_rank_gloo_combine_equals_single_run():
    import oracle
    from paper_2210_15874_gb300 import workloads as W

    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    w = W.qaoa_workload("shard_n6", 6, 2, index=11, trajectories=50, batch=50, p1=0.02, p2=0.05, damping=0.05)
    gates, G = oracle.qaoa_gates(w.n, w.edges, w.gammas, w.betas)
    full = oracle.traj_run(w.n, w.edges, gates, G, oracle.make_noise(**w.noise_kwargs()), w.seed, 0, 50,
                           want_amps=False)
    K = 50
    mean = full["s1"] / K
    se = np.sqrt(max(0.0, full["s2"] / K - mean * mean) / K)
    for rank in range(world):
        m, s, probs = out[rank]
        assert abs(m - mean) < 1e-12 and abs(s - se) < 1e-12
        np.testing.assert_allclose(probs, full["probs_sum"] / K, atol=1e-14)

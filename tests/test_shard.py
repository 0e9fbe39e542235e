"""Host logic of the multi-rank batched run (CPU only).

* the LPT split covers every instance exactly once and its makespan is within
  (4/3 - 1/(3m)) of the optimum found by brute force on small cost lists;
* two gloo ranks each solve their shard of a small batch (with the oracle standing in for
  the device solve) and the gathered results equal solving every instance on one rank;
* a rank that loses an instance, or two ranks that claim one, is an error on the host.
"""
import itertools
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2012_12419_gb300 import inputs, shard


def _opt_makespan(costs, m):
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


def test_lpt_partition_and_bound():
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(1, 4))
        costs = list(rng.integers(1, 100, size=n).astype(float))
        sh = shard.lpt_shards(costs, m)
        assert len(sh) == m
        assert sorted(i for s in sh for i in s) == list(range(n))
        span = max(sum(costs[i] for i in s) for s in sh)
        assert span <= (4 / 3 - 1 / (3 * m)) * _opt_makespan(costs, m) + 1e-9


def test_costs_follow_size_and_discount():
    p = dict(H=3, C=3, Q=4, gamma=0.9)
    q = dict(p, gamma=0.99)
    r = dict(p, C=4)
    assert shard.instance_cost(q) > shard.instance_cost(p)
    assert shard.instance_cost(r) > shard.instance_cost(p)
    ps = inputs.batch_params(512, seed=2)
    sh = shard.lpt_shards([shard.instance_cost(x) for x in ps], 4)
    loads = [sum(shard.instance_cost(ps[i]) for i in s) for s in sh]
    assert max(loads) / min(loads) < 1.05


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir, ps):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx, mine = shard.shard_of(ps, rank, world)
    local = {}
    for i, p in zip(idx, mine):
        V, pi, _, _ = oracle.solve(p, tol=1e-10)
        local[i] = (V.tolist(), pi.tolist())
    allres = shard.gather_by_index(local, len(ps))
    if rank == 0:
        with open(os.path.join(outdir, "gathered.npy"), "wb") as fh:
            np.save(fh, np.array([np.array(v[0]) for v in allres], dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def _small_batch():
    ps = []
    for k, (H, C, Q, g) in enumerate([(1, 1, 1, 0.9), (2, 1, 2, 0.95), (1, 2, 3, 0.99), (2, 2, 1, 0.9),
                                      (1, 1, 4, 0.95), (2, 1, 1, 0.99)]):
        ps.append(inputs.make_params(H, C, Q, g, seed=100 + k))
    return ps


def test_two_gloo_ranks_gather_every_instance():
    import torch.multiprocessing as mp

    ps = _small_batch()
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d, ps), nprocs=2, join=True, start_method="spawn")
        with open(os.path.join(d, "gathered.npy"), "rb") as fh:
            got = np.load(fh, allow_pickle=True)
    import oracle

    assert len(got) == len(ps)
    for p, v in zip(ps, got):
        V, _, _, _ = oracle.solve(p, tol=1e-10)
        assert np.array_equal(np.asarray(v, dtype=float), V)


def _lost_main(rank, world, port, outdir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    msgs = []
    for local in ({0: 1} if rank == 0 else {}, {0: 1, 1: 2} if rank == 0 else {1: 3}):
        try:
            shard.gather_by_index(local, 2)
            msgs.append("ok")
        except RuntimeError as e:
            msgs.append(str(e))
    with open(os.path.join(outdir, f"r{rank}.txt"), "w") as fh:
        fh.write("\n".join(msgs))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_rejects_missing_and_duplicate_instances():
    import torch.multiprocessing as mp

    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_lost_main, args=(2, _free_port(), d), nprocs=2, join=True, start_method="spawn")
        for r in range(2):
            lines = open(os.path.join(d, f"r{r}.txt")).read().splitlines()
            assert "solved on no rank" in lines[0]
            assert "solved on two ranks" in lines[1]


def test_shard_rejects_zero_ranks():
    with pytest.raises(ValueError):
        shard.lpt_shards([1.0], 0)

"""Host logic of the multi-GPU runs, on two CPU ranks over gloo.

Each rank works on its own seeded instance (replicas of one system) or on its
round-robin share of a batch of systems; the ranks meet only at the barrier
around the timed region and in the maximum of the elapsed times, from which
rank 0 forms the whole-job rate.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

WORLD = 2


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(WORLD), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    from paper_2403_01007_gb300 import replicas
    from paper_2403_01007_gb300 import synthetic as syn

    r, w, local = replicas.rank_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        inst = replicas.instance_of(r)
        eps, L = syn.workload_system(syn.SMALL, instance=inst)
        replicas.barrier()
        ms = 10.0 + 5.0 * r                      # rank 1 is the slow one
        ms_max = replicas.max_over_ranks(ms)
        rate = replicas.whole_job_rate(4 * 6, w, ms_max)
        # a batch of independent systems dealt to the ranks
        import torch
        mine = replicas.shard(syn.batch_instances(), r, w)
        n = torch.tensor([float(sum(x.nstates for x in mine)), float(len(mine))],
                         dtype=torch.float64)
        dist.all_reduce(n)
        seeds = sorted(x.seed for x in mine)
        replicas.barrier()
        out.put((r, w, local, inst, float(np.sum(eps)), float(np.sum(L[:3])), ms_max, rate,
                 n.tolist(), seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(WORLD)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [x[0] for x in res] == [0, 1]
    assert all(x[1] == WORLD and x[2] == x[0] for x in res)
    # distinct seeded instances per rank
    assert res[0][3] != res[1][3]
    assert (res[0][4], res[0][5]) != (res[1][4], res[1][5])
    # every rank sees the slowest rank's time and the same whole-job rate
    assert all(x[6] == 15.0 for x in res)
    expect = WORLD * 24 / 0.015
    assert all(x[7] == pytest.approx(expect) for x in res)
    # the shards of the batch are disjoint and together the whole batch
    from paper_2403_01007_gb300 import synthetic as syn
    batch = syn.batch_instances()
    total = [float(sum(x.nstates for x in batch)), float(len(batch))]
    assert all(x[8] == total for x in res)
    s0, s1 = set(res[0][9]), set(res[1][9])
    assert not (s0 & s1) and (s0 | s1) == {x.seed for x in batch}
    assert abs(len(s0) - len(s1)) <= 1


def test_single_rank_defaults(monkeypatch):
    from paper_2403_01007_gb300 import replicas
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.rank_env() == (0, 1, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)


def test_shard_rules():
    from paper_2403_01007_gb300 import replicas
    items = list(range(11))
    parts = [replicas.shard(items, r, 4) for r in range(4)]
    assert sorted(sum(parts, [])) == items
    assert [len(p) for p in parts] == [3, 3, 3, 2]
    assert replicas.shard(items, 0, 1) == items
    with pytest.raises(ValueError):
        replicas.shard(items, 4, 4)

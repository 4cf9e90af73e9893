"""Several ranks on the CPU (gloo, world size 2): the host logic of the multi-GPU path.

Roots are independent, so a graph's root order splits into contiguous shards,
one per rank, whose (count, hash, nodes, bytes) add up to the whole graph. Here
the CPU oracle computes each rank's shard (it stands in for the GPU, which this
machine does not have) and the library's own helpers split and combine; the
bench's max-over-ranks timing reduction runs on the same group.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    import paper_2401_05039_gb300 as m
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.workload("er200x300")
        live = np.nonzero(np.diff(g.u_off) > 0)[0].astype(np.int32)
        order = live[np.argsort(-np.diff(g.u_off)[live], kind="stable")]
        b, e = m.shard_bounds(len(order), rank, world)
        rows = oracle.per_root(g, roots=order[b:e], nthreads=1)
        mine = (int(rows[:, 0].sum()), int(rows[:, 1].sum(dtype=np.uint64)), int(rows[:, 2].sum()),
                int(rows[:, 3].sum()))
        tot = m.allreduce_totals(mine)
        slowest = bench.max_over_ranks(10.0 + rank, dist)
        q.put((rank, tot, slowest, e - b))
    finally:
        dist.destroy_process_group()


def _lpt_rank_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle.learn as learn
    import paper_2401_05039_gb300 as m
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.workload("er200x300")
        raw, _ = learn.root_features(g)  # the same raw values mbe_root_features computes on the GPU
        cost = m.static_root_cost(raw)
        mine = m.lpt_shards(cost, world)[rank]
        rows = oracle.per_root(g, roots=mine, nthreads=1)
        part = (int(rows[:, 0].sum()), int(rows[:, 1].sum(dtype=np.uint64)), int(rows[:, 2].sum()),
                int(rows[:, 3].sum()))
        tot = m.allreduce_totals(part)
        q.put((rank, tot, float(cost[mine].sum()), sorted(mine.tolist())))
    finally:
        dist.destroy_process_group()


def test_lpt_shards_balance_cost_and_add_up_over_two_gloo_ranks():
    # cost-balanced sharding: each rank runs its LPT share of the roots as an
    # explicit execution order; the shards partition the non-isolated roots,
    # their results add up to the whole graph, and the largest predicted load
    # is within LPT's bound
    import oracle.learn as learn
    import paper_2401_05039_gb300 as m
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_rank_main, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(WORLD)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = synth.workload("er200x300")
    whole = oracle.enumerate_graph(g)
    for rank, tot, _, _ in out:
        assert tot == tuple(whole), rank
    roots = sorted(sum((o[3] for o in out), []))
    assert roots == np.nonzero(np.diff(g.u_off) > 0)[0].tolist()
    cost = m.static_root_cost(learn.root_features(g)[0])
    loads = [o[2] for o in out]
    total, biggest = float(cost.sum()), float(cost.max())
    assert max(loads) <= total / WORLD + biggest
    assert max(loads) <= 4.0 / 3.0 * max(total / WORLD, biggest) + 1e-9


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_shards_bound(world):
    import paper_2401_05039_gb300 as m
    rng = np.random.default_rng(world)
    cost = np.concatenate([rng.pareto(1.5, 500) * 10, np.zeros(20)])
    shards = m.lpt_shards(cost, world)
    got = np.sort(np.concatenate(shards))
    assert got.tolist() == np.nonzero(cost > 0)[0].tolist()
    loads = [cost[s].sum() for s in shards]
    lower = max(cost.sum() / world, cost.max())
    assert max(loads) <= 4.0 / 3.0 * lower + 1e-9
    for s in shards:
        assert (np.diff(cost[s]) <= 0).all()


def test_shards_add_up_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(WORLD)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = oracle.enumerate_graph(synth.workload("er200x300"))
    sizes = sorted(o[3] for o in out)
    assert sizes[1] - sizes[0] <= 1
    for rank, tot, slowest, _ in out:
        assert tot == tuple(whole), rank
        assert slowest == 10.0 + (WORLD - 1)


@pytest.mark.parametrize("n,world", [(0, 1), (5, 1), (5, 2), (7, 3), (2, 4), (18849, 8)])
def test_shard_bounds_cover_once(n, world):
    import paper_2401_05039_gb300 as m
    spans = [m.shard_bounds(n, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    for (b0, e0), (b1, e1) in zip(spans, spans[1:]):
        assert e0 == b1
    sizes = [e - b for b, e in spans]
    assert max(sizes) - min(sizes) <= 1

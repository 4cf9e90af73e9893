"""GPU parity of the pruned search (iMBE's L - L' removal, Section II-C).

The pruned kernel variant against the oracle's pruned mode, bit-exact in
count, hash, nodes and algorithmic bytes (and the biclique set where it is
written); the oracle's pruned mode is pinned to the plain mode's sets and
to hand traces in test_oracle.py.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle.make_golden import expected_count
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbe():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2401_05039_gb300 as m
    m.load()
    return m


def gpu_tuple(r):
    return (int(r.count), int(r.hash), int(r.nodes), int(r.bytes_alg))


# both search frame layouts (1 = rows, 2 = columns)
LAYOUTS = [1, 2]


def run(mbe, g, **kw):
    G = mbe.Graph.from_synth(g)
    try:
        return G.enumerate(prune=1, **kw)
    finally:
        G.close()


def pruned(g, **kw):
    return oracle.enumerate_graph(g, prune=True, **kw)


def random_cases(seed, n, max_expected=3000):
    # several 32-row tiles with ragged tails; rows of one to five words
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        nU = int(rng.integers(1, 120))
        nV = int(rng.integers(1, 300))
        p = float(rng.choice([0.02, 0.05, 0.1, 0.2, 0.35, 0.5]))
        if expected_count(nU, nV, p) <= max_expected:
            out.append(H.random_graph(rng, nU, nV, p))
    return out


def twin_cases(seed, n):
    # long runs of equal counts and many twins: frames whose twin search
    # spans several 32-position chunks, with one- and multi-word rows
    # (densities and noise kept where the biclique count stays in the
    # thousands: denser rows with more noise reach 10^5 and beyond)
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nU = int(rng.integers(20, 300))
        nV = int(rng.integers(10, 200))
        out.append(H.twin_graph(rng, nU, nV, int(rng.integers(2, 16)), float(rng.choice([0.1, 0.2])),
                                float(rng.choice([0.0, 0.002, 0.006]))))
    return out


@pytest.mark.parametrize("layout", LAYOUTS)
def test_er200x300_full_set(mbe, layout):
    import torch
    g = synth.workload("er200x300")
    c, h, n, b, rec = pruned(g, records=True)
    assert n < oracle.enumerate_graph(g)[2]
    G = mbe.Graph.from_synth(g)
    buf = mbe.Bicliques.allocate(200000, 10000)
    r = G.enumerate(emit=1, bicliques=buf.buf, prune=1, layout=layout)
    torch.cuda.synchronize()
    assert gpu_tuple(r) == (c, h, n, b)
    assert sorted(buf.records()) == sorted(rec)
    # the per-root rows of the pruned run (a removed root has a zero row)
    pr = oracle.per_root(g, nthreads=4, prune=True)
    out = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
    G.enumerate(per_root=out, prune=1, layout=layout)
    assert (out.cpu().numpy().view(np.uint64) == pr).all()
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("seed", range(3))
def test_random_graphs(mbe, seed, layout):
    for g in random_cases(5000 + seed, 30):
        assert gpu_tuple(run(mbe, g, layout=layout)) == pruned(g), (g.nU, g.nV, g.nE)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("seed", range(3))
def test_twin_rich_graphs(mbe, seed, layout):
    for g in twin_cases(6000 + seed, 12):
        exp = pruned(g)
        assert gpu_tuple(run(mbe, g, layout=layout)) == exp, (g.nU, g.nV, g.nE)
        # the result does not depend on work stealing or the launch shape
        assert gpu_tuple(run(mbe, g, layout=layout, steal=0)) == exp
        assert gpu_tuple(run(mbe, g, layout=layout, blocks_per_sm=1, block_threads=64)) == exp


@pytest.mark.parametrize("layout", LAYOUTS)
def test_closed_forms(mbe, layout):
    g = H.complete(7, 9)
    for _ in range(4):
        g = H.disjoint_union(g, H.complete(7, 9))
    r = run(mbe, g, layout=layout)
    assert (r.count, r.nodes) == (5, 5)
    r = run(mbe, H.crown(12), layout=layout)
    assert r.count == 2 ** 12 - 2 and gpu_tuple(r) == pruned(H.crown(12))


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("min_r,min_l", [(2, 1), (1, 3), (3, 2)])
def test_size_filter(mbe, min_r, min_l, layout):
    for g in random_cases(7000 + 10 * min_r + min_l, 10) + twin_cases(7100 + min_r, 4):
        exp = pruned(g, min_r=min_r, min_l=min_l)
        assert gpu_tuple(run(mbe, g, layout=layout, min_r=min_r, min_l=min_l)) == exp, (g.nU, g.nV)


def test_output_full_and_shards(mbe):
    import torch
    g = synth.workload("er200x300")
    c, h, n, b, rec = pruned(g, records=True)
    G = mbe.Graph.from_synth(g)
    small = mbe.Bicliques.allocate(1000, 100)
    r = G.enumerate(emit=1, bicliques=small.buf, prune=1, check=False)
    torch.cuda.synchronize()
    assert r.status == 5 and gpu_tuple(r) == (c, h, n, b)
    assert small.buf.n_bicliques_written == c
    got = list(G.iter_bicliques(capacity_ids=4000, capacity_bicliques=400, prune=1))
    assert sorted(got) == sorted(rec)
    G.close()


def _golden(golden_dir, name):
    path = os.path.join(golden_dir, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle values for {name}")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_planted5k_whole_graph(mbe, golden_dir, layout):
    import torch
    gold = _golden(golden_dir, "planted5k_prune")
    g = synth.workload("planted5k")
    assert g.digest() == gold["graph"]["digest"]
    G = mbe.Graph.from_synth(g)
    out = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
    r = G.enumerate(per_root=out, prune=1, layout=layout)
    got = out.cpu().numpy().view(np.uint64)
    t = gold["total"]
    assert gpu_tuple(r) == (t["count"], int(t["hash"], 16), t["nodes"], t["bytes"])
    for root, row in gold["per_root"].items():
        assert tuple(int(x) for x in got[int(root)]) == (row["count"], int(row["hash"], 16), row["nodes"],
                                                         row["bytes"]), root
    G.close()


def test_chunglu200k_whole_graph(mbe, golden_dir):
    # the pruned whole-graph oracle total of the 200k x 1M Chung-Lu workload,
    # and its stored per-root rows (the column layout, as chosen automatically)
    import torch
    gold = _golden(golden_dir, "chunglu200k_prune")
    g = synth.workload("chunglu200k")
    assert g.digest() == gold["graph"]["digest"]
    G = mbe.Graph.from_synth(g)
    out = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
    r = G.enumerate(per_root=out, prune=1)
    got = out.cpu().numpy().view(np.uint64)
    t = gold["total"]
    assert gpu_tuple(r) == (t["count"], int(t["hash"], 16), t["nodes"], t["bytes"])
    for root, row in gold["per_root"].items():
        assert tuple(int(x) for x in got[int(root)]) == (row["count"], int(row["hash"], 16), row["nodes"],
                                                         row["bytes"]), root
    G.close()


def test_sampled_roots_of_the_large_workloads(mbe):
    # per-root rows of seeded random roots, oracle run live
    import torch
    for name, k in [("chunglu20k", 120), ("chunglu200k", 200)]:
        g = synth.workload(name)
        live = np.nonzero(np.diff(g.u_off) > 0)[0]
        roots = np.sort(np.random.default_rng(31).choice(live, size=k, replace=False)).astype(np.int32)
        exp = oracle.per_root(g, roots=roots, nthreads=8, prune=True)
        G = mbe.Graph.from_synth(g)
        out = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
        r = G.enumerate(per_root=out, prune=1)
        got = out.cpu().numpy().view(np.uint64)[roots]
        assert (got == exp).all(), name
        assert int(out[:, 0].sum()) == r.count
        # the same bicliques as the plain search
        p = G.enumerate()
        assert (r.count, r.hash) == (p.count, p.hash) and r.nodes < p.nodes
        G.close()


def test_root_above_the_bitset_limit_is_unsupported(mbe):
    for kw in ({}, {"bitset_max_words": 1}):
        g = H.complete(3, 2100) if not kw else H.complete(3, 100)
        with pytest.raises(mbe.MBEError) as e:
            run(mbe, g, **kw)
        assert e.value.status == 8


def test_batch(mbe, golden_dir):
    # the batched form, pruned: every graph's totals equal the oracle's
    # pruned run (random, twin-rich and small planted graphs of several size
    # classes, in one call)
    rng = np.random.default_rng(77)
    graphs = random_cases(8000, 20) + twin_cases(8001, 10) + [H.complete(5, 7), H.crown(9)]
    graphs += [H.random_graph(rng, 150, 600, 0.02) for _ in range(4)]
    for layout in (0, 1, 2):
        per, tot = mbe.enumerate_batch(synth.pack(graphs), prune=1, layout=layout)
        exp = [pruned(g) for g in graphs]
        assert [gpu_tuple(p) for p in per] == exp, layout
        assert tot.count == sum(e[0] for e in exp) and tot.nodes == sum(e[2] for e in exp)

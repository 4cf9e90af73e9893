"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so the bar is bit-exact: count, hash, nodes and algorithmic
bytes equal the oracle's, and on small graphs the sorted biclique set too.
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

# both search frame layouts (1 = rows, 2 = columns): the result must not depend on the layout
LAYOUTS = [1, 2]


@pytest.fixture(scope="module")
def mbe():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2401_05039_gb300 as m
    m.load()
    return m


def run(mbe, g, **kw):
    G = mbe.Graph.from_synth(g)
    try:
        r = G.enumerate(**kw)
    finally:
        G.close()
    return r


def oracle_tuple(g):
    return oracle.enumerate_graph(g)


def gpu_tuple(r):
    return (int(r.count), int(r.hash), int(r.nodes), int(r.bytes_alg))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_er200x300_full_set(mbe, golden_dir, layout):
    import torch
    g = synth.workload("er200x300")
    with open(os.path.join(golden_dir, "er200x300.json")) as f:
        gold = json.load(f)
    assert g.digest() == gold["graph"]["digest"]
    c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
    G = mbe.Graph.from_synth(g)
    buf = mbe.Bicliques.allocate(200000, 10000)
    r = G.enumerate(emit=1, bicliques=buf.buf, layout=layout)
    torch.cuda.synchronize()
    assert gpu_tuple(r) == (c, h, n, b)
    got = raw_records(buf)
    assert len(got) == c
    assert all(ascending(R) and ascending(L) for R, L in got)
    assert sorted(got) == sorted(rec)
    G.close()


def raw_records(buf):
    """The records as the library wrote them (no sorting here): [(R, L), ...]."""
    n = int(buf.buf.n_bicliques_written)
    ids = buf.ids.cpu().numpy()
    out = []
    for o in buf.offsets[:n].cpu().numpy().tolist():
        nr, nl = int(ids[o]), int(ids[o + 1])
        out.append((tuple(ids[o + 2:o + 2 + nr].tolist()), tuple(ids[o + 2 + nr:o + 2 + nr + nl].tolist())))
    return out


def ascending(t):
    return all(x < y for x, y in zip(t, t[1:]))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_output_full_keeps_exact_totals_and_reports_sizes(mbe, layout):
    # a buffer that is too small: the call returns MBE_ERR_OUTPUT_FULL with
    # count, hash, nodes and bytes still equal to the oracle's, and the sizes
    # the whole output needs; a second call with those sizes returns every
    # biclique, each written as R ascending then L ascending
    import torch
    g = synth.workload("er200x300")
    c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
    need_ids = sum(2 + len(R) + len(L) for R, L in rec)
    G = mbe.Graph.from_synth(g)
    for cap_ids, cap_bic in [(200000, 100), (1000, 10000), (0, 0)]:
        small = mbe.Bicliques.allocate(cap_ids, cap_bic)
        r = G.enumerate(emit=1, bicliques=small.buf, layout=layout, check=False)
        torch.cuda.synchronize()
        assert r.status == 5, (cap_ids, cap_bic)
        assert gpu_tuple(r) == (c, h, n, b)
        assert small.buf.n_bicliques_written == c
        assert small.buf.n_ids_written == need_ids
    full = mbe.Bicliques.allocate(need_ids, c)
    r = G.enumerate(emit=1, bicliques=full.buf, layout=layout)
    torch.cuda.synchronize()
    assert r.status == 0 and gpu_tuple(r) == (c, h, n, b)
    assert full.buf.n_ids_written == need_ids and full.buf.n_bicliques_written == c
    got = raw_records(full)
    assert all(ascending(R) and ascending(L) for R, L in got)
    assert sorted(got) == sorted(rec)
    G.close()


def _random_cases(seed, n, max_expected=3000):
    # sizes spanning several 32-row tiles with ragged tails; densities whose
    # Bernoulli expected biclique count keeps the oracle at milliseconds
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        nU = int(rng.integers(1, 120))
        nV = int(rng.integers(1, 300))
        p = float(rng.choice([0.02, 0.05, 0.1, 0.2, 0.35, 0.5]))
        if expected_count(nU, nV, p) <= max_expected:
            out.append(H.random_graph(rng, nU, nV, p))
    return out


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("layout", LAYOUTS)
def test_random_graphs_vs_oracle(mbe, seed, layout):
    for g in _random_cases(1000 + seed, 30):
        assert gpu_tuple(run(mbe, g, layout=layout)) == oracle_tuple(g), (g.nU, g.nV, g.nE)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_wide_rows_multiword(mbe, layout):
    # degrees near 90, 315 and 1100 give rows of 2, 5 and 18 words
    rng = np.random.default_rng(7)
    for nU, nV, p in [(16, 200, 0.45), (12, 700, 0.45), (12, 2000, 0.55)]:
        g = H.random_graph(rng, nU, nV, p)
        assert gpu_tuple(run(mbe, g, layout=layout)) == oracle_tuple(g), (nV, p)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_closed_forms(mbe, layout):
    for a, b in [(1, 1), (3, 200), (70, 5), (40, 130)]:
        r = run(mbe, H.complete(a, b), layout=layout)
        assert r.count == 1 and r.nodes == a
    for n in [1, 33, 100]:
        assert run(mbe, H.matching(n), layout=layout).count == n
    for n in [3, 6, 10, 13]:
        r = run(mbe, H.crown(n), layout=layout)
        assert r.count == 2 ** n - 2
        assert gpu_tuple(r) == oracle_tuple(H.crown(n))
    r = run(mbe, H.empty(10, 10), layout=layout)
    assert (r.count, r.hash, r.nodes) == (0, 0, 0)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_emit_matches_closure(mbe, layout):
    import torch
    rng = np.random.default_rng(9)
    g = H.random_graph(rng, 60, 140, 0.15)
    G = mbe.Graph.from_synth(g)
    buf = mbe.Bicliques.allocate(500000, 50000)
    r = G.enumerate(emit=1, bicliques=buf.buf, layout=layout)
    torch.cuda.synchronize()
    got = buf.decode()
    adj = H.adjacency_sets(g)
    assert len(got) == r.count == len(set(got))
    assert all(H.is_closed_pair(g, R, L, adj) for R, L in got)
    assert oracle.biclique_hash(got) == r.hash
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_emit_records_sorted_on_wide_sides(mbe, layout):
    # sides longer than a warp (the radix-sort path of the R merge) and long
    # L sides: the records equal the oracle's, each side already ascending
    import torch
    graphs = [H.complete(70, 5), H.complete(3, 200), H.crown(9),
              synth.planted(600, 700, 0.02, 6, (30, 60), (8, 14), 0.3, 5),
              H.random_graph(np.random.default_rng(12), 16, 700, 0.45)]
    for g in graphs:
        c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
        need = sum(2 + len(R) + len(L) for R, L in rec)
        G = mbe.Graph.from_synth(g)
        buf = mbe.Bicliques.allocate(need, c)
        r = G.enumerate(emit=1, bicliques=buf.buf, layout=layout)
        torch.cuda.synchronize()
        got = raw_records(buf)
        assert gpu_tuple(r) == (c, h, n, b), g.name
        assert all(ascending(R) and ascending(L) for R, L in got), g.name
        assert sorted(got) == sorted(rec), g.name
        G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_options_do_not_change_result(mbe, layout):
    g = synth.workload("er200x300")
    base = gpu_tuple(run(mbe, g, layout=layout))
    assert base == oracle_tuple(g)
    for kw in [dict(steal=0), dict(block_threads=32, blocks_per_sm=1), dict(block_threads=1024, blocks_per_sm=1),
               dict(block_threads=128, blocks_per_sm=4)]:
        assert gpu_tuple(run(mbe, g, layout=layout, **kw)) == base, kw


@pytest.mark.parametrize("layout", LAYOUTS)
def test_explicit_orders_and_shards(mbe, layout):
    import torch
    g = synth.workload("er200x300")
    base = oracle_tuple(g)
    live = np.nonzero(np.diff(g.u_off) > 0)[0].astype(np.int32)
    rng = np.random.default_rng(3)
    for order in [live, live[::-1].copy(), rng.permutation(live)]:
        t = torch.from_numpy(np.ascontiguousarray(order)).cuda()
        assert gpu_tuple(run(mbe, g, exec_order=t, n_exec=len(order), layout=layout)) == base
    # shards of the execution order add up
    G = mbe.Graph.from_synth(g)
    n = len(live)
    parts = [G.enumerate(root_begin=b, root_end=e, layout=layout) for b, e in [(0, 37), (37, 120), (120, n)]]
    tot = (sum(p.count for p in parts), sum(p.hash for p in parts) % (1 << 64), sum(p.nodes for p in parts),
           sum(p.bytes_alg for p in parts))
    assert tot == base
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_per_root_matches_oracle(mbe, layout):
    import torch
    g = synth.workload("er200x300")
    pr = oracle.per_root(g, nthreads=4)
    G = mbe.Graph.from_synth(g)
    buf = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
    G.enumerate(per_root=buf, layout=layout)
    got = buf.cpu().numpy().view(np.uint64)
    assert (got == pr).all()
    G.close()


def _golden(golden_dir, name):
    path = os.path.join(golden_dir, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle values for {name}")
    with open(path) as f:
        return json.load(f)


def _check_per_root_rows(mbe, g, gold, **kw):
    import torch
    G = mbe.Graph.from_synth(g)
    buf = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
    r = G.enumerate(per_root=buf, **kw)
    got = buf.cpu().numpy().view(np.uint64)
    for root, row in gold["per_root"].items():
        u = int(root)
        exp = (row["count"], int(row["hash"], 16), row["nodes"], row["bytes"])
        assert tuple(int(x) for x in got[u]) == exp, (u, exp)
    G.close()
    return r, got


@pytest.mark.parametrize("layout", LAYOUTS)
def test_planted5k_totals(mbe, golden_dir, layout):
    gold = _golden(golden_dir, "planted5k")
    g = synth.workload("planted5k")
    assert g.digest() == gold["graph"]["digest"], "generator drew a different graph on this machine"
    r, got = _check_per_root_rows(mbe, g, gold, layout=layout)
    t = gold["total"]
    assert gpu_tuple(r) == (t["count"], int(t["hash"], 16), t["nodes"], t["bytes"])
    assert int(got[:, 0].sum()) == t["count"]


@pytest.mark.parametrize("layout", LAYOUTS)
def test_chunglu20k_roots(mbe, golden_dir, layout):
    # per-root rows of a seeded uniform prefix of the roots (their exact sum
    # and individual rows); the whole-graph total when the oracle finished it
    gold = _golden(golden_dir, "chunglu20k")
    g = synth.workload("chunglu20k")
    assert g.digest() == gold["graph"]["digest"], "generator drew a different graph on this machine"
    r, got = _check_per_root_rows(mbe, g, gold, layout=layout)
    pre = gold["prefix"]
    live = np.nonzero(np.diff(g.u_off) > 0)[0]
    perm = np.random.default_rng(pre["seed"]).permutation(live)[:pre["k"]]
    s = got[perm].sum(axis=0, dtype=np.uint64)
    exp = pre["sum"]
    # a sum stored without bytes was taken under an earlier byte model (its
    # per-root rows carry bytes and are checked above)
    nb = 4 if exp["bytes"] is not None else 3
    assert tuple(int(x) for x in s[:nb]) == (exp["count"], int(exp["hash"], 16), exp["nodes"], exp["bytes"])[:nb]
    assert int(got[:, 0].sum()) == r.count and int(got[:, 2].sum()) == r.nodes
    if gold.get("total"):
        t = gold["total"]
        assert gpu_tuple(r)[:nb] == (t["count"], int(t["hash"], 16), t["nodes"], t["bytes"])[:nb]


@pytest.mark.parametrize("layout", LAYOUTS)
def test_chunglu200k_whole_graph(mbe, golden_dir, layout):
    # the 200k x 1M Chung-Lu workload: the whole-graph oracle total (count,
    # hash, nodes, bytes), its stored per-root rows (a seeded random sample,
    # the 100 heaviest roots and a sample of high-degree roots), and per-root
    # rows adding up to the total
    gold = _golden(golden_dir, "chunglu200k")
    g = synth.workload("chunglu200k")
    assert g.digest() == gold["graph"]["digest"]
    r, got = _check_per_root_rows(mbe, g, gold, layout=layout)
    assert int(got[:, 0].sum()) == r.count
    assert int(got[:, 2].sum()) == r.nodes
    t = gold["total"]
    assert t is not None
    assert gpu_tuple(r) == (t["count"], int(t["hash"], 16), t["nodes"], t["bytes"])


def test_invalid_layout_rejected(mbe):
    g = synth.workload("er200x300")
    G = mbe.Graph.from_synth(g)
    for bad in (-1, 3):
        assert G.enumerate(layout=bad, check=False).status == 1  # MBE_ERR_INVALID_ARG
    assert gpu_tuple(G.enumerate(layout=0)) == oracle_tuple(g)
    G.close()


def wide_graphs():
    """Graphs with roots of degree above 2,048 (the widest bitset level set)."""
    rng = np.random.default_rng(5)
    edges = [(u, v) for u in range(3) for v in range(5000)]
    us, vs = np.nonzero(rng.random((40, 5000)) < 0.02)
    edges += [(3 + int(u), int(v)) for u, v in zip(us, vs)]
    k3 = H.graph(43, 5000, edges, "K3,5000 + 40 sparse vertices")
    rng = np.random.default_rng(6)
    edges = [(int(u), int(v)) for u, v in zip(*np.nonzero(rng.random((5, 6000)) < 0.9))]
    edges += [(5 + int(u), int(v)) for u, v in zip(*np.nonzero(rng.random((30, 6000)) < 0.01))]
    hubs = H.graph(35, 6000, edges, "5 hubs sharing ~4,900 neighbours + 30 sparse vertices")
    return [k3, hubs, H.complete(2, 2100),
            synth.chung_lu(200, 10000, 12000, 1.8, 2.5, 8000, 7),   # one root of degree 2,694
            synth.chung_lu(400, 15000, 20000, 1.9, 2.5, 8000, 8),   # 3,178
            synth.chung_lu(150, 12000, 15000, 1.7, 2.6, 10000, 9)]  # 2,057 and 4,494


@pytest.mark.parametrize("layout", LAYOUTS)
def test_wide_roots_take_the_sorted_list_path(mbe, layout):
    # roots (and, for the hub graph, nodes two and three levels down) wider
    # than 2,048 vertices run as sorted-list frames with reverse-scan counts;
    # narrower children become bitset frames. Bit-exact against the oracle,
    # including the per-root rows of the widest graph.
    import torch
    for g in wide_graphs():
        assert int(np.diff(g.u_off).max()) > 2048
        assert gpu_tuple(run(mbe, g, layout=layout)) == oracle_tuple(g), g.name
    g = wide_graphs()[-1]
    G = mbe.Graph.from_synth(g)
    buf = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
    G.enumerate(per_root=buf, layout=layout)
    assert (buf.cpu().numpy().view(np.uint64) == oracle.per_root(g, nthreads=4)).all()
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("words", [1, 2])
def test_bitset_limit_sweep(mbe, layout, words):
    # a bitset limit of 64 or 128 vertices sends every wider level set of
    # these small graphs through the list path (roots, inner nodes, list
    # children and bitset children of list nodes): results do not change
    import torch
    for g in _random_cases(2000 + words, 20):
        assert gpu_tuple(run(mbe, g, layout=layout, bitset_max_words=words)) == oracle_tuple(g), (g.nU, g.nV)
    g = synth.workload("er200x300")
    c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
    G = mbe.Graph.from_synth(g)
    buf = mbe.Bicliques.allocate(200000, 10000)
    r = G.enumerate(emit=1, bicliques=buf.buf, layout=layout, bitset_max_words=words)
    torch.cuda.synchronize()
    got = raw_records(buf)
    assert gpu_tuple(r) == (c, h, n, b)
    assert all(ascending(R) and ascending(L) for R, L in got)
    assert sorted(got) == sorted(rec)
    assert gpu_tuple(G.enumerate(layout=layout, bitset_max_words=words, steal=0)) == (c, h, n, b)
    G.close()


def test_invalid_graphs_rejected(mbe):
    g = H.random_graph(np.random.default_rng(1), 10, 12, 0.4)
    bad = g.u_adj.copy()
    seg = slice(int(g.u_off[2]), int(g.u_off[3]))
    if bad[seg].size >= 2:
        bad[seg] = bad[seg][::-1]
    with pytest.raises(mbe.MBEError) as e:
        mbe.Graph(g.nU, g.nV, g.u_off, bad, g.v_off, g.v_adj)
    assert e.value.status == 2
    vadj = g.v_adj.copy()
    vadj[0] = (vadj[0] + 1) % g.nU
    with pytest.raises(mbe.MBEError) as e:
        mbe.Graph(g.nU, g.nV, g.u_off, g.u_adj, g.v_off, vadj)
    assert e.value.status == 2


@pytest.mark.parametrize("layout", LAYOUTS)
def test_arena_overflow_is_reported_then_recovers(mbe, layout):
    g = synth.workload("er200x300")
    G = mbe.Graph.from_synth(g)
    r = G.enumerate(arena_bytes=256, check=False, layout=layout)
    assert r.status == 4  # MBE_ERR_ARENA_FULL, no hang, no fault
    r2 = G.enumerate(layout=layout)
    assert gpu_tuple(r2) == oracle_tuple(g)
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_watchdog_expires_cleanly(mbe, layout):
    # one worker holds the single heavy root while the others wait for work;
    # a 1 ms watchdog makes their wait run out: the call returns
    # MBE_ERR_TIMEOUT, and the next call with the default watchdog succeeds
    g = H.crown(18)
    G = mbe.Graph.from_synth(g)
    r = G.enumerate(watchdog_ms=1, steal=0, check=False, layout=layout)
    assert r.status == 6
    r2 = G.enumerate(layout=layout)
    assert r2.status == 0 and r2.count == 2 ** 18 - 2
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("min_r,min_l", [(1, 2), (2, 1), (3, 4), (2, 2)])
def test_size_filter_matches_oracle(mbe, layout, min_r, min_l):
    # (|R| >= min_r, |L| >= min_l)-filtered enumeration: count, hash, nodes and
    # bytes equal the oracle's filtered run (which is pinned to the plain set
    # filtered by size), on random graphs, a wide graph (sorted-list path) and
    # with the bicliques written
    import torch
    kw = dict(layout=layout, min_r=min_r, min_l=min_l)
    for g in _random_cases(3000 + 10 * min_r + min_l, 12) + [wide_graphs()[1]]:
        assert gpu_tuple(run(mbe, g, **kw)) == oracle.enumerate_graph(g, min_r=min_r, min_l=min_l), (g.nU, g.nV)
    g = synth.workload("er200x300")
    c, h, n, b, rec = oracle.enumerate_graph(g, records=True, min_r=min_r, min_l=min_l)
    G = mbe.Graph.from_synth(g)
    buf = mbe.Bicliques.allocate(200000, 10000)
    r = G.enumerate(emit=1, bicliques=buf.buf, **kw)
    torch.cuda.synchronize()
    got = raw_records(buf)
    assert gpu_tuple(r) == (c, h, n, b)
    assert sorted(got) == sorted(rec) and all(len(R) >= min_r and len(L) >= min_l for R, L in got)
    # the batch path applies the same filter per graph
    sub = [H.random_graph(np.random.default_rng(k), 40, 90, 0.2) for k in range(6)]
    per, tot = mbe.enumerate_batch(synth.pack(sub), **kw)
    for x, p in zip(sub, per):
        assert gpu_tuple(p) == oracle.enumerate_graph(x, min_r=min_r, min_l=min_l)
    G.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_bicliques_to_pinned_host_memory_in_shards(mbe, layout):
    # the kernels write the records straight into pinned host buffers; with a
    # buffer far smaller than the output, the shard iterator splits the root
    # order until every shard fits, and the shards' records are exactly the
    # oracle's set (size filter included)
    import torch
    g = synth.workload("er200x300")
    _, _, _, _, rec = oracle.enumerate_graph(g, records=True)
    G = mbe.Graph.from_synth(g)
    buf = mbe.Bicliques.allocate(200000, 10000, pinned_host=True)
    r = G.enumerate(emit=1, bicliques=buf.buf, layout=layout)
    torch.cuda.synchronize()
    assert r.count == len(rec) and sorted(buf.records()) == sorted(rec)
    got = list(G.iter_bicliques(capacity_ids=4000, capacity_bicliques=400, layout=layout))
    assert sorted(got) == sorted(rec)
    got = list(G.iter_bicliques(capacity_ids=4000, capacity_bicliques=400, layout=layout, min_r=2, min_l=3))
    assert sorted(got) == sorted(oracle.enumerate_graph(g, records=True, min_r=2, min_l=3)[4])
    G.close()

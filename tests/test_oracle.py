"""Pins for the CPU oracle: it is checked against things other than itself.

- SplitMix64 against the published output sequence of seed 0;
- Algorithm 1 against hand traces (count, nodes, bytes, the biclique set);
- closed forms (complete, matching, crown, star, empty, disjoint union);
- an independent brute-force closure enumerator on >= 1,000 random graphs,
  itself pinned by the crown graph's 2^n - 2;
- invariants: closure of every emitted pair, side swap, relabelling,
  per-root decomposition;
- the pruned mode (iMBE's L - L' removal) against its own hand traces, a
  closed form (disjoint twin blocks) and the plain mode's biclique sets.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import helpers as H

MASK = (1 << 64) - 1


def sm_hash(pairs):
    """Digest of (R, L) pairs: U ids tagged 2u, V ids tagged 2v+1."""
    return oracle.biclique_hash(pairs)


# ----------------------------------------------------------------- SplitMix64

def test_splitmix64_published_sequence():
    # SplitMix64 with state 0 (Steele, Lea & Flood 2014; Vigna's splitmix64.c):
    # the k-th output is SM(k * 0x9e3779b97f4a7c15) with the gamma added first.
    gamma = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    got = [oracle.sm((k * gamma) & MASK) for k in range(4)]
    assert got == expect


def test_sm_zero_not_fixed_point():
    # the gamma is added before the mix, so vertex 0 of U still contributes
    assert oracle.sm(0) != 0


# ------------------------------------------------------------------ hand traces

def _traces(golden_dir):
    with open(os.path.join(golden_dir, "hand_traces.json")) as f:
        return json.load(f)["traces"]


def test_hand_traces(golden_dir):
    for t in _traces(golden_dir):
        g = H.graph(t["nU"], t["nV"], t["edges"])
        c, h, n, b, bb, rec = oracle.enumerate_graph(g, records=True, bytes_b=True)
        expect = [(tuple(r), tuple(l)) for r, l in t["bicliques"]]
        assert c == t["count"], t["name"]
        assert n == t["nodes"], t["name"]
        assert b == t["bytes"], t["name"]
        assert bb == t["bytes_b"], t["name"]
        # the per-root driver adds up to the same two byte counts
        pr = oracle.per_root(g, bytes_b=True)
        assert int(pr[:, 3].sum()) == b and int(pr[:, 4].sum()) == bb, t["name"]
        assert H.canon(rec) == H.canon(expect), t["name"]
        assert h == sm_hash(expect)


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("a,b", [(1, 1), (1, 5), (4, 1), (3, 7), (9, 4), (16, 16)])
def test_complete_bipartite_one_biclique(a, b):
    g = H.complete(a, b)
    c, h, n, byt, rec = oracle.enumerate_graph(g, records=True)
    assert c == 1
    assert rec == [(tuple(range(a)), tuple(range(b)))]
    assert h == sm_hash(rec)
    # every U vertex is popped once at the top level; only the first is maximal
    assert n == a
    # each top-level node reads N(x) and the b lists N(w) of length a
    assert byt == a * 4 * (b + b * a)
    # no node below the top level: the second byte model counts the same
    assert oracle.enumerate_graph(g, bytes_b=True)[4] == byt


@pytest.mark.parametrize("n", [1, 2, 5, 40])
def test_perfect_matching(n):
    g = H.matching(n)
    c, h, nodes, _, rec = oracle.enumerate_graph(g, records=True)
    assert c == n and nodes == n
    assert H.canon(rec) == [((i,), (i,)) for i in range(n)]


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8, 10])
def test_crown_graph(n):
    # every nonempty proper subset S of U pairs with V minus the matched copies of S
    g = H.crown(n)
    c, h, _, _, rec = oracle.enumerate_graph(g, records=True)
    assert c == 2 ** n - 2
    expect = []
    for mask in range(1, 2 ** n - 1):
        S = tuple(i for i in range(n) if mask >> i & 1)
        expect.append((S, tuple(v for v in range(n) if v not in S)))
    assert H.canon(rec) == H.canon(expect)
    assert h == sm_hash(expect)


def test_star_graphs():
    assert oracle.enumerate_graph(H.complete(1, 9))[0] == 1
    c, h, n, _ = oracle.enumerate_graph(H.complete(9, 1))
    assert c == 1 and n == 9


def test_empty_and_isolated():
    assert oracle.enumerate_graph(H.empty(0, 0))[:3] == (0, 0, 0)
    assert oracle.enumerate_graph(H.empty(5, 7))[:3] == (0, 0, 0)
    # isolated vertices on either side change nothing
    g = H.graph(6, 6, [(0, 0), (0, 1), (1, 0), (1, 1)])
    c, h, n, _, rec = oracle.enumerate_graph(g, records=True)
    assert c == 1 and rec == [((0, 1), (0, 1))] and n == 2


def test_figure1_fact():
    # Section II-A: with K_{3,3} on {A,B,C} x {F,G,H}, ({A,B,C},{F,G,H}) is
    # maximal and ({A,B},{F,G,H}) is not. U = A..E -> 0..4, V = F..K -> 0..5;
    # the extra edges touch no whole side of the block.
    edges = [(u, v) for u in range(3) for v in range(3)] + [(3, 0), (3, 3), (4, 4), (4, 5), (0, 5)]
    g = H.graph(5, 6, edges)
    _, _, _, _, rec = oracle.enumerate_graph(g, records=True)
    assert ((0, 1, 2), (0, 1, 2)) in rec
    assert ((0, 1), (0, 1, 2)) not in rec


def test_disjoint_union_adds():
    rng = np.random.default_rng(5)
    g1 = H.random_graph(rng, 12, 15, 0.3)
    g2 = H.random_graph(rng, 9, 20, 0.25)
    r1 = oracle.enumerate_graph(g1, records=True)
    r2 = oracle.enumerate_graph(g2, records=True)
    ru = oracle.enumerate_graph(H.disjoint_union(g1, g2), records=True)
    assert ru[0] == r1[0] + r2[0]
    shifted = [(tuple(u + g1.nU for u in r), tuple(v + g1.nV for v in l)) for r, l in r2[4]]
    assert H.canon(ru[4]) == H.canon(r1[4] + shifted)
    assert ru[1] == (r1[1] + sm_hash(shifted)) & MASK


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("n", [2, 3, 5, 8, 11])
def test_bruteforce_crown(n):
    c, h, rec = oracle.bruteforce(H.crown(n), records=True)
    assert c == 2 ** n - 2
    assert all(len(r) + len(l) == n for r, l in rec)


def test_bruteforce_complete_and_matching():
    assert oracle.bruteforce(H.complete(5, 8))[0] == 1
    assert oracle.bruteforce(H.matching(12))[0] == 12
    assert oracle.bruteforce(H.empty(4, 4))[0] == 0


def test_mbea_matches_bruteforce_random():
    rng = np.random.default_rng(20240110)
    n_graphs = 0
    for trial in range(1100):
        nU = int(rng.integers(1, 13))
        nV = int(rng.integers(1, 40))
        p = float(rng.choice([0.05, 0.15, 0.3, 0.5, 0.7, 0.9]))
        g = H.random_graph(rng, nU, nV, p)
        c1, h1, _, _, rec1 = oracle.enumerate_graph(g, records=True)
        c2, h2, rec2 = oracle.bruteforce(g, records=True)
        assert c1 == c2 and h1 == h2, (trial, nU, nV, p)
        assert H.canon(rec1) == H.canon(rec2), trial
        n_graphs += 1
    assert n_graphs >= 1000


def test_mbea_matches_bruteforce_swapped_sides():
    # |V| small, |U| large: brute force over the V side of the swapped graph
    rng = np.random.default_rng(77)
    for trial in range(150):
        nU = int(rng.integers(10, 60))
        nV = int(rng.integers(1, 12))
        g = H.random_graph(rng, nU, nV, float(rng.choice([0.1, 0.3, 0.6])))
        _, _, _, _, rec = oracle.enumerate_graph(g, records=True)
        _, _, recT = oracle.bruteforce(g.swapped(), records=True)
        assert H.canon(rec) == H.canon([(l, r) for r, l in recT]), trial


# ------------------------------------------------------------------- invariants

def test_every_pair_closed_and_unique():
    rng = np.random.default_rng(3)
    for _ in range(40):
        g = H.random_graph(rng, int(rng.integers(5, 40)), int(rng.integers(5, 60)), 0.2)
        _, _, _, _, rec = oracle.enumerate_graph(g, records=True)
        adj = H.adjacency_sets(g)
        assert len(set(H.canon(rec))) == len(rec)
        for r, l in rec:
            assert H.is_closed_pair(g, r, l, adj)


def test_side_swap_same_set():
    rng = np.random.default_rng(11)
    for _ in range(30):
        g = H.random_graph(rng, int(rng.integers(5, 30)), int(rng.integers(5, 30)), 0.25)
        c, h, _, _, rec = oracle.enumerate_graph(g, records=True)
        cT, hT, _, _, recT = oracle.enumerate_graph(g.swapped(), records=True)
        assert c == cT
        assert H.canon(rec) == H.canon([(l, r) for r, l in recT])


def test_relabelling_invariance():
    rng = np.random.default_rng(12)
    for _ in range(30):
        g = H.random_graph(rng, int(rng.integers(5, 35)), int(rng.integers(5, 35)), 0.2)
        pu, pv = rng.permutation(g.nU), rng.permutation(g.nV)
        c, h, _, _, rec = oracle.enumerate_graph(g, records=True)
        c2, h2, _, _, rec2 = oracle.enumerate_graph(H.relabel(g, pu, pv), records=True)
        mapped = [(tuple(int(pu[u]) for u in r), tuple(int(pv[v]) for v in l)) for r, l in rec]
        assert c == c2 and H.canon(rec2) == H.canon(mapped) and h2 == sm_hash(mapped)


def test_per_root_decomposition():
    import synth
    rng = np.random.default_rng(13)
    graphs = [H.random_graph(rng, 30, 40, 0.15), synth.workload("er200x300")]
    for g in graphs:
        total = oracle.enumerate_graph(g)
        pr = oracle.per_root(g, nthreads=2)
        assert int(pr[:, 0].sum()) == total[0]
        assert int(pr[:, 1].sum(dtype=np.uint64)) == total[1]
        assert int(pr[:, 2].sum()) == total[2]
        assert int(pr[:, 3].sum()) == total[3]
        # isolated vertices are never popped
        iso = np.nonzero(np.diff(g.u_off) == 0)[0]
        assert (pr[iso] == 0).all()


def test_root_order_is_degree_then_id():
    rng = np.random.default_rng(14)
    g = H.random_graph(rng, 50, 20, 0.2)
    seq = oracle.root_order(g)
    deg = np.diff(g.u_off)
    keys = [(int(deg[u]), int(u)) for u in seq]
    assert keys == sorted(keys)
    assert set(seq.tolist()) == set(np.nonzero(deg > 0)[0].tolist())


def test_batch_driver_matches_serial():
    import synth
    gs = [synth.batch_graph(1000 + i, u_range=(16, 40), v_range=(16, 60)) for i in range(12)]
    b = synth.pack(gs)
    out = oracle.batch(b, nthreads=3)
    for i, g in enumerate(gs):
        assert tuple(int(x) for x in out[i]) == oracle.enumerate_graph(g)


# ------------------------------------------------------------ size filter

@pytest.mark.parametrize("min_r,min_l", [(1, 2), (2, 1), (2, 2), (3, 4), (5, 2)])
def test_size_filter_is_the_filtered_set(min_r, min_l):
    # the size-filtered enumeration returns exactly the maximal bicliques with
    # |R| >= min_r and |L| >= min_l (its pruning drops only subtrees and
    # candidates that cannot reach both sizes), with fewer or equal nodes;
    # on small graphs also against the brute-force closure enumeration
    rng = np.random.default_rng(100 * min_r + min_l)
    graphs = [synth.workload("er200x300"), H.crown(7), H.complete(4, 6)]
    graphs += [H.random_graph(rng, int(rng.integers(2, 12)), int(rng.integers(2, 30)), p) for p in (0.2, 0.4, 0.6)
               for _ in range(8)]
    for g in graphs:
        c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
        want = [(R, L) for R, L in rec if len(R) >= min_r and len(L) >= min_l]
        fc, fh, fn, fb, frec = oracle.enumerate_graph(g, records=True, min_r=min_r, min_l=min_l)
        assert H.canon(frec) == H.canon(want), g.name
        assert fc == len(want) and fh == sm_hash(want)
        assert fn <= n
        if g.nU <= 12:
            bc, bh, brec = oracle.bruteforce(g, records=True)
            assert H.canon([(R, L) for R, L in brec if len(R) >= min_r and len(L) >= min_l]) == H.canon(frec)
        pr = oracle.per_root(g, min_r=min_r, min_l=min_l)
        assert (int(pr[:, 0].sum()), int(pr[:, 1].sum(dtype=np.uint64)), int(pr[:, 2].sum()),
                int(pr[:, 3].sum())) == (fc, fh, fn, fb)


def test_size_filter_hand_trace():
    # path u0-v0-u1-v1-u2 (hand trace 1): with |L| >= 2 only ({u1}, {v0, v1})
    # passes; u0 and u2 (degree 1) are never popped, u1 is (one node)
    g = H.graph(3, 2, [(0, 0), (1, 0), (1, 1), (2, 1)])
    c, h, n, b, rec = oracle.enumerate_graph(g, records=True, min_l=2)
    assert rec == [((1,), (0, 1))] and (c, n) == (1, 1)
    # with |R| >= 2 both edges' bicliques pass, the star at u1 does not; all
    # three roots are popped (three nodes), none has a child
    c, h, n, b, rec = oracle.enumerate_graph(g, records=True, min_r=2)
    assert H.canon(rec) == [((0, 1), (0,)), ((1, 2), (1,))] and n == 3


# ------------------------------------------------------ pruned mode (iMBE)

def test_prune_hand_traces(golden_dir):
    with open(os.path.join(golden_dir, "prune_traces.json")) as f:
        traces = json.load(f)["traces"]
    for t in traces:
        g = H.graph(t["nU"], t["nV"], t["edges"])
        expect = H.canon([(tuple(r), tuple(l)) for r, l in t["bicliques"]])
        c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
        assert (c, n, b) == (t["count"], t["plain_nodes"], t["plain_bytes"]), t["name"]
        assert H.canon(rec) == expect
        c, h, n, b, rec = oracle.enumerate_graph(g, records=True, prune=True)
        assert (c, n, b) == (t["count"], t["pruned_nodes"], t["pruned_bytes"]), t["name"]
        assert H.canon(rec) == expect and h == sm_hash(expect)
        # the per-root driver prunes the top level the same way
        pr = oracle.per_root(g, prune=True)
        assert (int(pr[:, 0].sum()), int(pr[:, 2].sum()), int(pr[:, 3].sum())) == (c, n, b)
        assert sum(int(x) for x in pr[:, 1]) & MASK == h


@pytest.mark.parametrize("k,a,b", [(1, 5, 3), (3, 4, 2), (6, 1, 7), (2, 9, 9)])
def test_prune_twin_blocks_closed_form(k, a, b):
    # k disjoint copies of K_{a,b}: the a vertices of a block are twins, so
    # only the first of each block is popped (plain: all k*a are)
    g = H.complete(a, b)
    for _ in range(k - 1):
        g = H.disjoint_union(g, H.complete(a, b))
    assert oracle.enumerate_graph(g)[2] == k * a
    c, h, n, _ = oracle.enumerate_graph(g, prune=True)
    assert (c, n) == (k, k)


@pytest.mark.parametrize("n", [2, 5, 9])
def test_prune_no_twins_changes_nothing(n):
    # matching and crown graphs: no two U vertices share a neighbourhood in
    # any level set the search meets on the matching; the crown's top level
    # has none either
    g = H.matching(n)
    assert oracle.enumerate_graph(g, prune=True) == oracle.enumerate_graph(g)
    c, h, _, _ = oracle.enumerate_graph(H.crown(n), prune=True)
    assert c == 2 ** n - 2


def test_prune_same_bicliques_fewer_nodes_random():
    rng = np.random.default_rng(1401)
    fewer = 0
    for trial in range(400):
        nU = int(rng.integers(1, 13))
        nV = int(rng.integers(1, 30))
        p = float(rng.choice([0.1, 0.3, 0.5, 0.8]))
        g = H.random_graph(rng, nU, nV, p)
        c0, h0, n0, b0, rec0 = oracle.enumerate_graph(g, records=True)
        c1, h1, n1, b1, rec1 = oracle.enumerate_graph(g, records=True, prune=True)
        assert (c1, h1) == (c0, h0) and H.canon(rec1) == H.canon(rec0), trial
        assert H.canon(rec1) == H.canon(oracle.bruteforce(g, records=True)[2]), trial
        assert n1 <= n0 and b1 <= b0, trial
        fewer += n1 < n0
        # whole run = sum of its roots, pruned too
        pr = oracle.per_root(g, prune=True)
        assert int(pr[:, 0].sum()) == c1 and int(pr[:, 2].sum()) == n1 and int(pr[:, 3].sum()) == b1, trial
        assert (int(pr[:, 1].sum()) & MASK) == h1, trial
    assert fewer > 50


@pytest.mark.parametrize("min_r,min_l", [(2, 1), (1, 3), (2, 2)])
def test_prune_with_size_filter(min_r, min_l):
    rng = np.random.default_rng(99)
    for trial in range(60):
        g = H.random_graph(rng, int(rng.integers(2, 12)), int(rng.integers(2, 25)), 0.4)
        a = oracle.enumerate_graph(g, records=True, min_r=min_r, min_l=min_l)
        b = oracle.enumerate_graph(g, records=True, min_r=min_r, min_l=min_l, prune=True)
        assert a[:2] == b[:2] and H.canon(a[4]) == H.canon(b[4]) and b[2] <= a[2], trial

"""Small hand-built graphs and set utilities shared by the tests (no enumeration arithmetic)."""
from __future__ import annotations

import numpy as np

import synth


def graph(nU, nV, edges, name=""):
    edges = list(edges)
    eu = [e[0] for e in edges]
    ev = [e[1] for e in edges]
    return synth.from_edges(nU, nV, eu, ev, name)


def complete(a, b):
    return graph(a, b, [(u, v) for u in range(a) for v in range(b)], f"K{a},{b}")


def matching(n):
    return graph(n, n, [(i, i) for i in range(n)], f"M{n}")


def crown(n):
    """K_{n,n} minus a perfect matching."""
    return graph(n, n, [(u, v) for u in range(n) for v in range(n) if u != v], f"S{n}")


def empty(a, b):
    return graph(a, b, [], f"E{a},{b}")


def random_graph(rng, nU, nV, p):
    m = rng.random((nU, nV)) < p
    us, vs = np.nonzero(m)
    return graph(nU, nV, zip(us.tolist(), vs.tolist()), f"rand{nU}x{nV}")


def disjoint_union(g1, g2):
    e1 = edges_of(g1)
    e2 = [(u + g1.nU, v + g1.nV) for u, v in edges_of(g2)]
    return graph(g1.nU + g2.nU, g1.nV + g2.nV, e1 + e2, "union")


def edges_of(g):
    out = []
    for u in range(g.nU):
        for k in range(g.u_off[u], g.u_off[u + 1]):
            out.append((u, int(g.u_adj[k])))
    return out


def relabel(g, pu, pv):
    """Graph with U vertex u renamed pu[u] and V vertex v renamed pv[v]."""
    return graph(g.nU, g.nV, [(int(pu[u]), int(pv[v])) for u, v in edges_of(g)], g.name + "'")


def adjacency_sets(g):
    nu = [set() for _ in range(g.nU)]
    nv = [set() for _ in range(g.nV)]
    for u, v in edges_of(g):
        nu[u].add(v)
        nv[v].add(u)
    return nu, nv


def is_closed_pair(g, R, L, adj=None):
    """L = Gamma(R) and R = Gamma(L), both nonempty: the definition of a maximal biclique."""
    nu, nv = adj if adj is not None else adjacency_sets(g)
    if not R or not L:
        return False
    gR = set.intersection(*[nu[u] for u in R])
    gL = set.intersection(*[nv[v] for v in L])
    return gR == set(L) and gL == set(R)


def canon(pairs):
    return sorted((tuple(sorted(r)), tuple(sorted(l))) for r, l in pairs)


def twin_graph(rng, nU, nV, n_base, p, flip):
    """Each U vertex copies one of n_base random rows of density p and flips
    every bit with probability flip: many vertices share a neighbourhood,
    in G and (far more often) inside the level sets of a search."""
    base = rng.random((n_base, nV)) < p
    rows = base[rng.integers(0, n_base, size=nU)] ^ (rng.random((nU, nV)) < flip)
    us, vs = np.nonzero(rows)
    return graph(nU, nV, zip(us.tolist(), vs.tolist()), f"twins{nU}x{nV}")

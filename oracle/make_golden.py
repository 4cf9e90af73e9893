"""Write the stored expected values under tests/golden/ by running the CPU oracle.

Calls only ``oracle`` and the input generators in ``synth``; nothing here
touches the GPU library. Usage:

    python oracle/make_golden.py er200x300 planted5k chunglu20k chunglu200k batch4096 [--threads N]
    python oracle/make_golden.py planted5k --prune [--threads N]


Each workload writes ``tests/golden/<name>.json`` with the graph digest (so a
machine that draws a different graph is caught before parity is checked),
oracle totals where the oracle can finish the whole graph, and per-root
(count, hash, nodes, bytes) rows for a sample of roots. Hashes are written
as hex strings.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")


# Version of the algorithmic-byte model in oracle.bytes_node; progress files
# written under another version keep valid counts, hashes and nodes only.
BYTES_MODEL = 2


def _row(r, with_bytes=True):
    out = {"count": int(r[0]), "hash": hex(int(r[1])), "nodes": int(r[2])}
    out["bytes"] = int(r[3]) if with_bytes else None
    if len(r) > 4:
        out["bytes_b"] = int(r[4])  # the second byte model (bitset rows or reverse-scanned lists)
    return out


def _graph_info(g):
    deg = np.diff(g.u_off)
    return {"nU": g.nU, "nV": g.nV, "nE": g.nE, "digest": g.digest(), "max_deg_u": int(deg.max(initial=0)),
            "max_deg_v": int(np.diff(g.v_off).max(initial=0)), "isolated_u": int((deg == 0).sum())}


def _sample_roots(g, pr_full, n_heavy, n_random, seed):
    rng = np.random.default_rng(seed)
    live = np.nonzero(np.diff(g.u_off) > 0)[0]
    heavy = np.argsort(-pr_full[:, 2].astype(np.int64), kind="stable")[:n_heavy] if pr_full is not None else []
    rand = rng.choice(live, size=min(n_random, live.size), replace=False)
    return sorted(set(int(x) for x in heavy) | set(int(x) for x in rand))


def set_digest(records):
    """SHA-256 of the canonical (sorted) biclique list, R then L, both sorted."""
    canon = sorted((tuple(sorted(r)), tuple(sorted(l))) for r, l in records)
    h = hashlib.sha256()
    for r, l in canon:
        h.update(np.array([len(r), len(l)] + list(r) + list(l), dtype=np.int64).tobytes())
    return h.hexdigest()


def whole_graph(name, g, threads, n_heavy=16, n_random=48, records=False):
    t0 = time.time()
    pr = oracle.per_root(g, nthreads=threads, bytes_b=True)
    out = {"workload": name, "graph": _graph_info(g),
           "total": _row(pr.sum(axis=0, dtype=np.uint64)), "oracle_seconds": round(time.time() - t0, 1),
           "oracle_threads": threads}
    roots = _sample_roots(g, pr, n_heavy, n_random, seed=len(name))
    out["per_root"] = {str(r): _row(pr[r]) for r in roots}
    if records:
        c, h, n, b, rec = oracle.enumerate_graph(g, records=True)
        assert c == out["total"]["count"] and hex(h) == out["total"]["hash"]
        out["set_sha256"] = set_digest(rec)
    return out


def whole_graph_pruned(name, g, threads, n_heavy=16, n_random=48):
    """The pruned mode (iMBE's L - L' removal): whole-graph total and per-root rows."""
    t0 = time.time()
    pr = oracle.per_root(g, nthreads=threads, prune=True)
    out = {"workload": name, "mode": "pruned", "graph": _graph_info(g),
           "total": _row(pr.sum(axis=0, dtype=np.uint64)), "oracle_seconds": round(time.time() - t0, 1),
           "oracle_threads": threads}
    roots = _sample_roots(g, pr, n_heavy, n_random, seed=len(name) + 1)
    out["per_root"] = {str(r): _row(pr[r]) for r in roots}
    return out


def sampled_roots(name, g, threads, n_random=40, n_top_degree=8):
    """Per-root rows only (the whole graph is beyond the oracle's reach)."""
    t0 = time.time()
    deg = np.diff(g.u_off)
    rng = np.random.default_rng(len(name))
    live = np.nonzero(deg > 0)[0]
    rand = rng.choice(live, size=min(n_random, live.size), replace=False)
    # a few roots from the upper degree decile, to cover wide local universes
    upper = live[deg[live] >= np.quantile(deg[live], 0.9)]
    top = rng.choice(upper, size=min(n_top_degree, upper.size), replace=False)
    roots = np.array(sorted(set(rand.tolist()) | set(top.tolist())), dtype=np.int32)
    pr = oracle.per_root(g, roots=roots, nthreads=threads, bytes_b=True)
    return {"workload": name, "graph": _graph_info(g), "total": None,
            "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": threads,
            "per_root": {str(int(r)): _row(pr[i]) for i, r in enumerate(roots)}}


def expected_count(nU, nV, p, a_max=128, b_max=512):
    """Expected number of maximal bicliques of a Bernoulli(p) bipartite graph (selection proxy only).

    Sum over side sizes (a, b) of C(nU,a) C(nV,b) p^(ab) (1-p^a)^(nV-b) (1-p^b)^(nU-a), truncated to
    a <= a_max, b <= b_max where the terms are negligible for the densities used here.
    """
    if p <= 0 or nU == 0 or nV == 0:
        return 0.0
    from scipy.special import gammaln
    a = np.arange(1, min(nU, a_max) + 1, dtype=np.float64)[:, None]
    b = np.arange(1, min(nV, b_max) + 1, dtype=np.float64)[None, :]
    lp = math.log(p)
    lc_a = gammaln(nU + 1) - gammaln(a + 1) - gammaln(nU - a + 1)
    lc_b = gammaln(nV + 1) - gammaln(b + 1) - gammaln(nV - b + 1)
    qa = -np.expm1(a * lp)
    qb = -np.expm1(b * lp)
    with np.errstate(divide="ignore"):
        e = lc_a + lc_b + a * b * lp + (nV - b) * np.log(qa) + (nU - a) * np.log(qb)
    return float(np.exp(np.clip(e, -745, 700)).sum())


def batch(name, threads, n_graphs=4096, budget_count=2.0e5, n_heavy_graphs=12, roots_per_heavy=6):
    """Oracle over the graphs whose expected count is below budget_count; root samples of heavy ones."""
    t0 = time.time()
    gs = [synth.batch_graph(3 + i) for i in range(n_graphs)]
    est = []
    for g in gs:
        p = g.nE / max(g.nU * g.nV, 1)
        est.append(expected_count(g.nU, g.nV, p))
    est = np.array(est)
    chosen = [i for i in range(n_graphs) if est[i] <= budget_count]
    sub = synth.pack([gs[i] for i in chosen])
    order = np.argsort(-est[chosen], kind="stable").astype(np.int32)
    res = oracle.batch(sub, nthreads=threads, order=order)
    per_graph = {str(i): dict(_row(res[k]), nU=gs[i].nU, nV=gs[i].nV, nE=gs[i].nE)
                 for k, i in enumerate(chosen)}
    heavy = [int(i) for i in np.argsort(-est)[:n_heavy_graphs]]
    heavy_roots = {}
    for i in heavy:
        g = gs[i]
        rng = np.random.default_rng(i)
        live = np.nonzero(np.diff(g.u_off) > 0)[0]
        roots = np.sort(rng.choice(live, size=min(roots_per_heavy, live.size), replace=False)).astype(np.int32)
        pr = oracle.per_root(g, roots=roots, nthreads=threads)
        heavy_roots[str(i)] = {str(int(r)): _row(pr[k]) for k, r in enumerate(roots)}
    digests = hashlib.sha256("".join(g.digest() for g in gs).encode()).hexdigest()[:32]
    return {"workload": name, "n_graphs": n_graphs, "digest_of_digests": digests,
            "selection": f"graphs whose Bernoulli expected maximal-biclique count is <= {budget_count:g}",
            "n_selected": len(chosen), "expected_count_total": float(est.sum()),
            "per_graph": per_graph, "heavy_graph_roots": heavy_roots,
            "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": threads}


def batch_rest_roots(path, threads, back=(2, 16, 48)):
    """Per-root rows for the batch graphs the oracle cannot finish whole.

    For every graph of the batch without a stored whole-graph row, the
    top-level candidates at pop positions n - b for b in `back` (n = number
    of non-isolated roots): the last pops have the smallest subtrees, so
    these rows stay within seconds of oracle time each while still covering
    nodes below the top level. Added to the existing batch golden in place.
    """
    with open(path) as f:
        gold = json.load(f)
    t0 = time.time()
    done = set(int(k) for k in gold["per_graph"])
    rest = [i for i in range(gold["n_graphs"]) if i not in done]
    out = {}
    for i in rest:
        g = synth.batch_graph(3 + i)
        seq = oracle.root_order(g)
        n = len(seq)
        roots = np.array(sorted({int(seq[n - b]) for b in back if n - b >= 0}), dtype=np.int32)
        pr = oracle.per_root(g, roots=roots, nthreads=threads)
        out[str(i)] = {str(int(r)): _row(pr[k]) for k, r in enumerate(roots)}
    gold["rest_graph_roots"] = out
    gold["rest_graph_roots_about"] = ("graphs without a whole-graph oracle row: per-root rows of the top-level pops at "
                                      f"positions n - {', n - '.join(str(b) for b in back)} of the (degree, id) order")
    gold["rest_oracle_seconds"] = round(time.time() - t0, 1)
    with open(path, "w") as f:
        json.dump(gold, f, indent=1, sort_keys=True)
    return len(out)


def prefix_sample(name, g, threads, seed=20240110, batch=256, keep_rows=300, progress=None, time_budget=None):
    """Per-root oracle rows for the roots in a seeded random order, in batches, resumable.

    Progress is saved after every batch to `progress` (a .npz). The stored
    golden covers the first K roots of the permutation: their summed
    (count, hash, nodes, bytes) and `keep_rows` individual rows. When K is
    every root, the sum is the whole-graph total.
    """
    rng = np.random.default_rng(seed)
    live = np.nonzero(np.diff(g.u_off) > 0)[0]
    perm = rng.permutation(live).astype(np.int32)
    rows = np.zeros((0, 5), dtype=np.uint64)
    model = BYTES_MODEL
    if progress and os.path.exists(progress):
        d = np.load(progress)
        # rows without the second byte model's column are not resumed
        if int(d["seed"]) == seed and d["digest"].item() == g.digest() and d["rows"].shape[1] == 5:
            rows = d["rows"]
            model = int(d["bytes_model"]) if "bytes_model" in d else 1
    t0 = time.time()
    # heaviest roots of a batch first (two-hop volume), so that no thread is
    # left alone with a late heavy root; the rows keep the permutation order
    deg_v = np.diff(g.v_off)
    volume = np.array([int(deg_v[g.u_adj[g.u_off[r]:g.u_off[r + 1]]].sum()) for r in range(g.nU)], dtype=np.int64)
    while rows.shape[0] < perm.size and (time_budget is None or time.time() - t0 < time_budget):
        k = rows.shape[0]
        roots = perm[k:k + batch]
        heavy = np.argsort(-volume[roots], kind="stable")
        part = np.empty((roots.size, 5), dtype=np.uint64)
        part[heavy] = oracle.per_root(g, roots=roots[heavy], nthreads=threads, bytes_b=True)
        rows = np.concatenate([rows, part])
        if progress:
            np.savez(progress + ".tmp.npz", rows=rows, seed=seed, digest=np.array(g.digest()),
                     bytes_model=np.array(model))
            os.replace(progress + ".tmp.npz", progress)
        print(f"{name}: {rows.shape[0]}/{perm.size} roots, {time.time() - t0:.0f}s", flush=True)
    K = rows.shape[0]
    pick = np.random.default_rng(seed + 1).choice(K, size=min(keep_rows, K), replace=False) if K else []
    pick = sorted(int(x) for x in pick)
    total = rows.sum(axis=0, dtype=np.uint64) if K else np.zeros(5, np.uint64)
    fresh = model == BYTES_MODEL
    if not fresh and pick:
        # rows from an older byte model: the kept rows are run again, whole
        again = oracle.per_root(g, roots=perm[pick], nthreads=threads, bytes_b=True)
        assert (again[:, :3] == rows[pick, :3]).all(), "count/hash/nodes changed between oracle versions"
        rows = rows.copy()
        rows[pick] = again
    return {"workload": name, "graph": _graph_info(g), "total": _row(total, fresh) if K == perm.size else None,
            "prefix": {"seed": seed, "k": int(K), "n_roots": int(perm.size), "sum": _row(total, fresh),
                       "about": "sum over the first k roots of the seeded permutation of the non-isolated U vertices"
                                + ("" if fresh else "; bytes not stored: the sum was taken under an earlier byte model")},
            "per_root": {str(int(perm[i])): _row(rows[i]) for i in pick},
            "oracle_threads": threads}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--prefix", action="store_true", help="resumable seeded-order per-root run (large graphs)")
    ap.add_argument("--progress", default=None, help="progress file for --prefix")
    ap.add_argument("--budget", type=float, default=None, help="seconds to spend in this --prefix invocation")
    ap.add_argument("--batch", type=int, default=256, help="roots per oracle call in --prefix mode")
    ap.add_argument("--prune", action="store_true", help="the pruned mode: writes <name>_prune.json")
    ap.add_argument("--batch-rest", action="store_true",
                    help="add per-root rows of the batch graphs without whole-graph rows to batch4096.json")
    args = ap.parse_args()
    os.makedirs(GOLDEN, exist_ok=True)
    if args.batch_rest:
        n = batch_rest_roots(os.path.join(GOLDEN, "batch4096.json"), args.threads)
        print(f"batch4096: per-root rows for {n} graphs", flush=True)
        return
    for name in args.names:
        t0 = time.time()
        suffix = ""
        if args.prune:
            out = whole_graph_pruned(name, synth.workload(name), args.threads)
            suffix = "_prune"
        elif args.prefix:
            out = prefix_sample(name, synth.workload(name), args.threads, batch=args.batch, progress=args.progress,
                                time_budget=args.budget)
        elif name == "er200x300":
            out = whole_graph(name, synth.workload(name), args.threads, n_heavy=8, n_random=24, records=True)
        elif name in ("planted5k", "chunglu20k"):
            out = whole_graph(name, synth.workload(name), args.threads)
        elif name == "chunglu200k":
            out = sampled_roots(name, synth.workload(name), args.threads)
        elif name == "batch4096":
            out = batch(name, args.threads)
        else:
            raise SystemExit(f"unknown workload {name}")
        path = os.path.join(GOLDEN, f"{name}{suffix}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
        print(f"{name}: wrote {path} in {time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main()

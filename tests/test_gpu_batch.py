"""Batched enumeration (many graphs, one call) against the stored CPU-oracle values."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbe():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    import paper_2401_05039_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def gold(golden_dir):
    with open(os.path.join(golden_dir, "batch4096.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def graphs(gold):
    gs = [synth.batch_graph(3 + i) for i in range(gold["n_graphs"])]
    import hashlib
    dig = hashlib.sha256("".join(g.digest() for g in gs).encode()).hexdigest()[:32]
    assert dig == gold["digest_of_digests"], "generator drew different graphs on this machine"
    return gs


def _row(r):
    return (int(r.count), int(r.hash), int(r.nodes), int(r.bytes_alg))


def _exp(d):
    return (d["count"], int(d["hash"], 16), d["nodes"], d["bytes"])


@pytest.mark.parametrize("layout", [0, 1, 2])
def test_batch_selected_graphs_match_oracle(mbe, gold, graphs, layout):
    # layout 0 = the automatic choice per class; 1 = rows, 2 = columns
    ids = sorted(int(k) for k in gold["per_graph"])
    b = synth.pack([graphs[i] for i in ids])
    per, tot = mbe.enumerate_batch(b, layout=layout)
    assert tot.status == 0
    for k, i in enumerate(ids):
        assert _row(per[k]) == _exp(gold["per_graph"][str(i)]), i
    assert tot.count == sum(int(p.count) for p in per)


@pytest.mark.parametrize("layout", [1, 2])
def test_batch_heavy_graph_roots(mbe, gold, graphs, layout):
    import torch
    for gi, rows in gold["heavy_graph_roots"].items():
        g = graphs[int(gi)]
        G = mbe.Graph.from_synth(g)
        buf = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
        G.enumerate(per_root=buf, layout=layout)
        got = buf.cpu().numpy().view(np.uint64)
        G.close()
        for root, d in rows.items():
            assert tuple(int(x) for x in got[int(root)]) == _exp(d), (gi, root)


def test_batch_equals_single_graph_calls_and_autotune(mbe, gold, graphs):
    # a mixed slice (cheap and heavier graphs of every class present): the
    # batch equals one mbe_enumerate per graph, with default and tuned params
    ids = list(range(0, 400, 3))
    sub = [graphs[i] for i in ids]
    b = synth.pack(sub)
    per, tot = mbe.enumerate_batch(b)
    for g, p in zip(sub, per):
        G = mbe.Graph.from_synth(g)
        assert _row(G.enumerate()) == _row(p)
        G.close()
    table = mbe.autotune_batch(b, sample_per_class=16)
    classes = {mbe.batch_class(g.nU, g.nV, g.nE) for g in sub}
    for c in classes:
        assert table[c].valid == 1 and table[c].block_threads > 0 and table[c].layout in (1, 2)
    per2, tot2 = mbe.enumerate_batch(b, class_params=table)
    assert [_row(p) for p in per2] == [_row(p) for p in per]


def test_full_batch_in_one_call(mbe, gold, graphs):
    # the 4,096-graph workload as stated, in one mbe_enumerate_batch call:
    # every graph the oracle finished whole is exact; every other graph equals
    # one mbe_enumerate on its own, whose per-root rows match the oracle's
    # stored rows for that graph; per-graph device times are the class times
    import torch
    b = synth.pack(graphs)
    per, tot = mbe.enumerate_batch(b)
    assert tot.status == 0
    for k, d in gold["per_graph"].items():
        assert _row(per[int(k)]) == _exp(d), k
    rest = gold["rest_graph_roots"]
    assert len(rest) + len(gold["per_graph"]) == len(graphs)
    for gi, rows in rest.items():
        g = graphs[int(gi)]
        G = mbe.Graph.from_synth(g)
        buf = torch.zeros((g.nU, 4), dtype=torch.int64, device="cuda")
        r = G.enumerate(per_root=buf)
        got = buf.cpu().numpy().view(np.uint64)
        G.close()
        assert _row(r) == _row(per[int(gi)]), gi
        for root, d in rows.items():
            assert tuple(int(x) for x in got[int(root)]) == _exp(d), (gi, root)
    assert tot.count == sum(int(p.count) for p in per)
    assert tot.hash == sum(int(p.hash) for p in per) % (1 << 64)
    classes = {}
    for g, p in zip(graphs, per):
        classes.setdefault(mbe.batch_class(g.nU, g.nV, g.nE), set()).add(round(p.device_ms, 6))
    assert all(len(v) == 1 and min(v) > 0 for v in classes.values())
    assert sum(min(v) for v in classes.values()) <= tot.device_ms * 1.01

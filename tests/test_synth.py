"""The input generators are deterministic: the same seed draws the same graph on every machine."""
import json
import os

import numpy as np

import synth


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, f"{name}.json")) as f:
        return json.load(f)


def test_er_digest_and_shape(golden_dir):
    g = synth.workload("er200x300")
    gold = _golden(golden_dir, "er200x300")["graph"]
    assert (g.nU, g.nV, g.nE) == (gold["nU"], gold["nV"], gold["nE"])
    assert g.digest() == gold["digest"]


def test_csr_csc_are_transposes():
    g = synth.workload("er200x300")
    rows = np.repeat(np.arange(g.nU), np.diff(g.u_off))
    cols = np.repeat(np.arange(g.nV), np.diff(g.v_off))
    a = set(zip(rows.tolist(), g.u_adj.tolist()))
    b = set(zip(g.v_adj.tolist(), cols.tolist()))
    assert a == b and len(a) == g.nE
    for u in range(g.nU):
        seg = g.u_adj[g.u_off[u]:g.u_off[u + 1]]
        assert (np.diff(seg) > 0).all()


def test_same_seed_same_graph():
    a = synth.batch_graph(17)
    b = synth.batch_graph(17)
    c = synth.batch_graph(18)
    assert a.digest() == b.digest() != c.digest()
    assert 16 <= a.nU <= 512 and 16 <= a.nV <= 2048


def test_chung_lu_exact_edges_and_cap():
    g = synth.chung_lu(2000, 5000, 20000, 2.1, 2.3, 150, 9)
    assert g.nE == 20000
    assert np.diff(g.u_off).max() <= 150 and np.diff(g.v_off).max() <= 150


def test_planted_blocks_present():
    g = synth.planted(300, 300, 0.0, 5, (4, 6), (5, 8), 0.3, 21)
    # no background: every edge comes from a planted complete block
    deg = np.diff(g.u_off)
    assert g.nE > 0 and deg.max() <= 5 * 8

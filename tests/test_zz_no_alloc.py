"""mbe_enumerate_noalloc against mbe_enumerate, through the C ABI, on the GPU.

The no-allocation entry point serves callers that cannot allocate device
memory (a framework that owns the device memory pool, or a latency-critical
loop that must not meet cudaMalloc/cudaFree): it takes the graph in the
caller's device arrays and uses a fixed scratch array inside the library.
Its results must equal the CPU oracle's and the regular entry point's, on
consecutive calls (the scratch array keeps the previous call's contents).
"""
import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _device_arrays(g):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
            for a in (g.u_off, g.u_adj, g.v_off, g.v_adj)]


def _tuple(r):
    return (int(r.count), int(r.hash), int(r.nodes), int(r.bytes_alg))


@pytest.fixture(scope="module")
def mbe():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    import paper_2401_05039_gb300 as m
    m.load()
    return m


def test_noalloc_matches_oracle_and_enumerate_twice(mbe):
    # two calls in a row on each graph: both equal the CPU oracle and the
    # regular entry point (the fixed array keeps the previous call's contents)
    import torch
    import oracle
    graphs = [synth.workload("er200x300"),
              H.random_graph(np.random.default_rng(41), 77, 150, 0.12),
              synth.planted(600, 700, 0.02, 6, (6, 10), (8, 14), 0.3, 5)]
    for g in graphs:
        exp = oracle.enumerate_graph(g)
        G = mbe.Graph.from_synth(g)
        ref = _tuple(G.enumerate())
        G.close()
        assert ref == exp, g.name
        d = _device_arrays(g)
        for call in range(2):
            r = mbe.enumerate_noalloc(g.nU, g.nV, *d)
            torch.cuda.synchronize()
            assert r.status == 0
            assert _tuple(r) == exp, (g.name, call)


def test_noalloc_rejects_invalid_graphs_and_bad_tensors(mbe):
    # an unsorted list and a CSR/CSC pair that are not transposes (ids in
    # range: the device checks see them) come back as MBE_ERR_INVALID_GRAPH;
    # tensors of the wrong type or length are refused before the call
    import torch
    g = H.random_graph(np.random.default_rng(1), 10, 12, 0.4)
    uo, ua, vo, va = _device_arrays(g)
    u = int(np.nonzero(np.diff(g.u_off) >= 2)[0][0])
    seg = slice(int(g.u_off[u]), int(g.u_off[u + 1]))
    bad = ua.clone()
    bad[seg] = torch.flip(bad[seg], [0])
    assert mbe.enumerate_noalloc(g.nU, g.nV, uo, bad, vo, va, check=False).status == 2
    bad_v = va.clone()
    bad_v[0] = (bad_v[0] + 1) % g.nU
    assert mbe.enumerate_noalloc(g.nU, g.nV, uo, ua, vo, bad_v, check=False).status == 2
    with pytest.raises(mbe.MBEError):
        mbe.enumerate_noalloc(g.nU, g.nV, uo.long(), ua, vo, va)
    with pytest.raises(mbe.MBEError):
        mbe.enumerate_noalloc(g.nU + 1, g.nV, uo, ua, vo, va)
    with pytest.raises(mbe.MBEError):
        mbe.enumerate_noalloc(g.nU, g.nV, uo.cpu(), ua, vo, va)
    # and the entry point still gives the oracle's result afterwards
    import oracle
    assert _tuple(mbe.enumerate_noalloc(g.nU, g.nV, uo, ua, vo, va)) == oracle.enumerate_graph(g)


def test_noalloc_rejects_graphs_beyond_its_scratch(mbe):
    g = synth.workload("chunglu20k")
    d = _device_arrays(g)
    r = mbe.enumerate_noalloc(g.nU, g.nV, *d, check=False)
    assert r.status == 8  # MBE_ERR_UNSUPPORTED: the workspace exceeds the 64 MiB array
    # and the entry point still works afterwards
    import oracle
    g2 = synth.workload("er200x300")
    assert _tuple(mbe.enumerate_noalloc(g2.nU, g2.nV, *_device_arrays(g2))) == oracle.enumerate_graph(g2)

"""Seeded synthetic bipartite graphs for tests and benchmarks.

Input infrastructure only: this package draws graphs and converts edge lists
to the CSR (U -> V) and CSC (V -> U) arrays that both the CPU oracle and the
GPU library consume. It contains none of the enumeration's arithmetic.

The five workloads stand in for the paper's KONECT datasets (Section IV,
Table I), which are not available: they reproduce the skewed, power-law,
community-rich structure the paper's evaluation describes, at sizes chosen
per workload (see ``WORKLOADS``).
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgraphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (gcc, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
            I64P = ctypes.POINTER(ctypes.c_int64)
            lib.gg_erdos_renyi.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                                           P32, P32, I64P]
            lib.gg_batch_graph.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_double), P32, P32, I64P]
            lib.gg_planted.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_uint64, P32, P32, I64P]
            lib.gg_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int32, ctypes.c_uint64, P32, P32, I64P]
            lib.gg_free.argtypes = [ctypes.c_void_p]
            for f in (lib.gg_erdos_renyi, lib.gg_batch_graph, lib.gg_planted, lib.gg_chung_lu):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Graph:
    """Bipartite graph G=(U,V,E) as CSR (U->V) and CSC (V->U), int32, sorted, no duplicates."""

    nU: int
    nV: int
    u_off: np.ndarray  # int32 [nU+1]
    u_adj: np.ndarray  # int32 [nE], V ids
    v_off: np.ndarray  # int32 [nV+1]
    v_adj: np.ndarray  # int32 [nE], U ids
    name: str = ""

    @property
    def nE(self) -> int:
        return int(self.u_adj.shape[0])

    def digest(self) -> str:
        """SHA-256 over sizes and CSR arrays (checks that two machines drew the same graph)."""
        h = hashlib.sha256()
        h.update(np.array([self.nU, self.nV, self.nE], dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(self.u_off, dtype=np.int32).tobytes())
        h.update(np.ascontiguousarray(self.u_adj, dtype=np.int32).tobytes())
        return h.hexdigest()[:32]

    def swapped(self) -> "Graph":
        """The same graph with the roles of U and V exchanged."""
        return Graph(self.nV, self.nU, self.v_off, self.v_adj, self.u_off, self.u_adj, self.name + "^T")


def from_edges(nU: int, nV: int, eu, ev, name: str = "") -> Graph:
    """Build sorted, de-duplicated CSR and CSC arrays from an edge list."""
    eu = np.asarray(eu, dtype=np.int64).ravel()
    ev = np.asarray(ev, dtype=np.int64).ravel()
    if eu.size:
        if eu.min() < 0 or eu.max() >= nU or ev.min() < 0 or ev.max() >= nV:
            raise ValueError("edge endpoint out of range")
    keys = np.unique(eu * max(nV, 1) + ev)
    u = (keys // max(nV, 1)).astype(np.int32)
    v = (keys % max(nV, 1)).astype(np.int32)
    u_off = np.zeros(nU + 1, dtype=np.int64)
    np.cumsum(np.bincount(u, minlength=nU), out=u_off[1:])
    order = np.lexsort((u, v))
    v_off = np.zeros(nV + 1, dtype=np.int64)
    np.cumsum(np.bincount(v, minlength=nV), out=v_off[1:])
    return Graph(nU, nV, u_off.astype(np.int32), v.copy(), v_off.astype(np.int32),
                 u[order].copy(), name)


def _take(eu_p, ev_p, ne) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    n = int(ne.value)
    eu = np.ctypeslib.as_array(eu_p, shape=(n,)).copy() if n else np.zeros(0, np.int32)
    ev = np.ctypeslib.as_array(ev_p, shape=(n,)).copy() if n else np.zeros(0, np.int32)
    lib.gg_free(ctypes.cast(eu_p, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(ev_p, ctypes.c_void_p))
    return eu, ev


def _ptrs():
    return ctypes.POINTER(ctypes.c_int32)(), ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int64()


def erdos_renyi(nU: int, nV: int, p: float, seed: int) -> Graph:
    """Bernoulli(p) per (u, v) pair, u-major; then random relabelling of both sides."""
    lib = _load()
    a, b, n = _ptrs()
    if lib.gg_erdos_renyi(nU, nV, p, seed, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)):
        raise MemoryError("gg_erdos_renyi failed")
    eu, ev = _take(a, b, n)
    return from_edges(nU, nV, eu, ev, f"er_{nU}x{nV}_p{p}_s{seed}")


def planted(nU: int, nV: int, p_bg: float, n_blocks: int, a_range, b_range, overlap: float,
            seed: int) -> Graph:
    """Bernoulli background plus overlapping planted complete blocks."""
    lib = _load()
    a, b, n = _ptrs()
    if lib.gg_planted(nU, nV, p_bg, n_blocks, a_range[0], a_range[1], b_range[0], b_range[1], overlap,
                      seed, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)):
        raise MemoryError("gg_planted failed")
    eu, ev = _take(a, b, n)
    return from_edges(nU, nV, eu, ev, f"planted_{nU}x{nV}_s{seed}")


def chung_lu(nU: int, nV: int, m: int, gamma_u: float, gamma_v: float, cap: int, seed: int) -> Graph:
    """Chung-Lu power-law bipartite graph with exactly m distinct edges and a degree cap."""
    lib = _load()
    a, b, n = _ptrs()
    if lib.gg_chung_lu(nU, nV, m, gamma_u, gamma_v, cap, seed, ctypes.byref(a), ctypes.byref(b),
                       ctypes.byref(n)):
        raise MemoryError("gg_chung_lu failed")
    eu, ev = _take(a, b, n)
    return from_edges(nU, nV, eu, ev, f"chunglu_{nU}x{nV}_m{m}_s{seed}")


def batch_graph(seed: int, u_range=(16, 512), v_range=(16, 2048), p_range=(0.02, 0.20)) -> Graph:
    """One graph of the many-small-graphs batch; its sizes and density come from its own seed."""
    lib = _load()
    nU, nV, p = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    a, b, n = _ptrs()
    if lib.gg_batch_graph(seed, u_range[0], u_range[1], v_range[0], v_range[1], p_range[0], p_range[1],
                          ctypes.byref(nU), ctypes.byref(nV), ctypes.byref(p), ctypes.byref(a),
                          ctypes.byref(b), ctypes.byref(n)):
        raise MemoryError("gg_batch_graph failed")
    eu, ev = _take(a, b, n)
    return from_edges(nU.value, nV.value, eu, ev, f"batch_s{seed}_p{p.value:.4f}")


@dataclass
class Batch:
    """Many graphs packed as concatenated CSR/CSC with per-graph offset tables."""

    nU: np.ndarray  # int32 [G]
    nV: np.ndarray  # int32 [G]
    edge_off: np.ndarray  # int64 [G+1], start of each graph's edges in u_adj/v_adj
    u_off: np.ndarray  # int32 [sum(nU)+G], each graph's CSR offsets (local, start at 0)
    v_off: np.ndarray  # int32 [sum(nV)+G]
    u_adj: np.ndarray  # int32 [E], local V ids
    v_adj: np.ndarray  # int32 [E], local U ids
    u_off_start: np.ndarray  # int64 [G], where graph g's u_off begins
    v_off_start: np.ndarray  # int64 [G]

    @property
    def n_graphs(self) -> int:
        return int(self.nU.shape[0])

    def graph(self, g: int) -> Graph:
        nu, nv = int(self.nU[g]), int(self.nV[g])
        e0, e1 = int(self.edge_off[g]), int(self.edge_off[g + 1])
        su, sv = int(self.u_off_start[g]), int(self.v_off_start[g])
        return Graph(nu, nv, self.u_off[su:su + nu + 1].copy(), self.u_adj[e0:e1].copy(),
                     self.v_off[sv:sv + nv + 1].copy(), self.v_adj[e0:e1].copy(), f"batch[{g}]")


def pack(graphs: list[Graph]) -> Batch:
    G = len(graphs)
    nU = np.array([g.nU for g in graphs], dtype=np.int32)
    nV = np.array([g.nV for g in graphs], dtype=np.int32)
    ne = np.array([g.nE for g in graphs], dtype=np.int64)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ne, out=edge_off[1:])
    u_off_start = np.zeros(G, dtype=np.int64)
    v_off_start = np.zeros(G, dtype=np.int64)
    if G:
        u_off_start[1:] = np.cumsum(nU.astype(np.int64) + 1)[:-1]
        v_off_start[1:] = np.cumsum(nV.astype(np.int64) + 1)[:-1]
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)  # noqa: E731
    return Batch(nU, nV, edge_off, cat([g.u_off for g in graphs], np.int32),
                 cat([g.v_off for g in graphs], np.int32), cat([g.u_adj for g in graphs], np.int32),
                 cat([g.v_adj for g in graphs], np.int32), u_off_start, v_off_start)


# ------------------------------------------------------------------ workloads
#
# The five seeded workloads. Sizes follow the evaluation's skewed power-law
# bipartite graphs (Section IV); the readings of under-specified details are
# stated next to each.

def workload(name: str, **kw):
    """Return the Graph (or Batch) for a named workload."""
    if name == "er200x300":
        # 200 x 300, Bernoulli(0.05) per pair, seed 0 (~3k edges)
        return erdos_renyi(200, 300, 0.05, 0)
    if name == "chunglu20k":
        # 20,000 x 50,000 Chung-Lu, 200,000 edges, exponents 2.1 / 2.3, degree cap 2,000, seed 1
        return chung_lu(20000, 50000, 200000, 2.1, 2.3, 2000, 1)
    if name == "planted5k":
        # 5,000 x 5,000, 1% background, 60 planted K_{15..25, 20..40}, 30% overlap, seed 2
        return planted(5000, 5000, 0.01, 60, (15, 25), (20, 40), 0.3, 2)
    if name == "batch4096":
        # 4,096 graphs, graph i drawn from seed 3+i
        n = kw.get("n_graphs", 4096)
        return pack([batch_graph(3 + i) for i in range(n)])
    if name == "chunglu200k":
        # 200,000 x 1,000,000 Chung-Lu, 5,000,000 edges, exponents 2.0 / 2.2, seed 4. The degree cap
        # is not given for this size; 400 keeps the hub core enumerable (with 2,000 the 320 x 320
        # hub block alone has density 0.45 and an estimated > 1e10 maximal bicliques).
        cap = kw.get("cap", 400)
        return chung_lu(200000, 1000000, 5000000, 2.0, 2.2, cap, 4)
    raise KeyError(name)


WORKLOADS = ("er200x300", "chunglu20k", "planted5k", "batch4096", "chunglu200k")

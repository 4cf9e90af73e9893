"""CPU oracle for maximal biclique enumeration (MBEA, paper Algorithm 1).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use it; the library's product path never
does. It shares no code with the GPU path.

``mbea_oracle.c`` holds the arithmetic (serial MBEA, per-root driver, batch
driver, brute-force closure enumerator, SplitMix64 hash); this module only
compiles it with gcc and marshals numpy arrays through ctypes. ``learn.py``
holds the per-root features, core numbers and the float64 reference of the
cost-model network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbea_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmbea_oracle.so")
_lib = None
_lock = threading.Lock()

_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U64P = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, portable flags, POSIX threads)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_sm.argtypes = [ctypes.c_uint64]
            lib.orc_sm.restype = ctypes.c_uint64
            lib.orc_enumerate.argtypes = [ctypes.c_int32, ctypes.c_int32, _I32P, _I32P, _I32P, _I32P, _U64P,
                                          ctypes.POINTER(_I32P), _I64P, _U64P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32]
            lib.orc_per_root.argtypes = [ctypes.c_int32, ctypes.c_int32, _I32P, _I32P, _I32P, _I32P, _I32P,
                                         ctypes.c_int64, _U64P, ctypes.c_int32, _U64P, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int32]
            lib.orc_root_order.argtypes = [ctypes.c_int32, _I32P, _I32P, _I64P]
            lib.orc_batch.argtypes = [ctypes.c_int32, _I32P, _I32P, _I64P, _I64P, _I64P, _I32P, _I32P, _I32P,
                                      _I32P, _I32P, _U64P, ctypes.c_int32]
            lib.orc_bruteforce.argtypes = [ctypes.c_int32, ctypes.c_int32, _I32P, _I32P, _U64P,
                                           ctypes.POINTER(_I32P), _I64P]
            lib.orc_free.argtypes = [ctypes.c_void_p]
            for f in (lib.orc_enumerate, lib.orc_per_root, lib.orc_root_order, lib.orc_batch, lib.orc_bruteforce):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_I32P)


def _c32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def sm(z: int) -> int:
    """One SplitMix64 output step of z (the hash primitive)."""
    return int(_load().orc_sm(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def _records(rec_p, n) -> list[tuple[tuple[int, ...], tuple[int, ...]]]:
    lib = _load()
    n = int(n.value)
    if n == 0:
        lib.orc_free(ctypes.cast(rec_p, ctypes.c_void_p))
        return []
    flat = np.ctypeslib.as_array(rec_p, shape=(n,)).tolist()
    lib.orc_free(ctypes.cast(rec_p, ctypes.c_void_p))
    out, i = [], 0
    while i < n:
        nr, nl = flat[i], flat[i + 1]
        r = tuple(flat[i + 2:i + 2 + nr])
        l = tuple(flat[i + 2 + nr:i + 2 + nr + nl])
        out.append((r, l))
        i += 2 + nr + nl
    return out


def _arrays(g):
    return _c32(g.u_off), _c32(g.u_adj), _c32(g.v_off), _c32(g.v_adj)


def enumerate_graph(g, records: bool = False, bytes_b: bool = False, min_r: int = 1, min_l: int = 1,
                    prune: bool = False):
    """Serial MBEA over the whole graph.

    Returns ``(count, hash, nodes, bytes)`` or, with ``records=True``,
    ``(count, hash, nodes, bytes, [(R, L), ...])`` with R, L sorted id tuples.
    ``bytes`` is the algorithmic byte count of the run; ``bytes_b=True``
    appends the count under the second byte model (bitset rows or reverse-
    scanned lists, whichever is cheaper per node). ``min_r``, ``min_l``: the
    size filter (only bicliques with |R| >= min_r and |L| >= min_l, and no
    search where none can pass). ``prune=True``: iMBE's L - L' removal
    (Section II-C): the same bicliques from fewer nodes; the second byte
    model is then not counted (0).
    """
    lib = _load()
    uo, ua, vo, va = _arrays(g)
    out = np.zeros(4, dtype=np.uint64)
    ob = np.zeros(1, dtype=np.uint64)
    rec_p, rec_n = _I32P(), ctypes.c_int64(0)
    rc = lib.orc_enumerate(g.nU, g.nV, _p32(uo), _p32(ua), _p32(vo), _p32(va), out.ctypes.data_as(_U64P),
                           ctypes.byref(rec_p) if records else None, ctypes.byref(rec_n) if records else None,
                           ob.ctypes.data_as(_U64P), int(min_r), int(min_l), int(bool(prune)))
    if rc:
        raise MemoryError("oracle enumeration failed")
    res = tuple(int(x) for x in out)
    if bytes_b:
        res = res + (int(ob[0]),)
    if records:
        return res + (_records(rec_p, rec_n),)
    return res


def per_root(g, roots=None, nthreads: int = 1, bytes_b: bool = False, min_r: int = 1, min_l: int = 1,
             prune: bool = False):
    """(count, hash, nodes, bytes) per top-level candidate; uint64 array [len(roots), 4].

    ``roots`` defaults to every U vertex (row u = vertex u). With
    ``bytes_b=True`` the rows have a fifth column: bytes under the second
    byte model. ``prune``: as in :func:`enumerate_graph` (a root that the
    pruning removes gets a zero row).
    """
    lib = _load()
    uo, ua, vo, va = _arrays(g)
    roots = np.arange(g.nU, dtype=np.int32) if roots is None else _c32(roots)
    out = np.zeros((roots.shape[0], 4), dtype=np.uint64)
    ob = np.zeros(max(roots.shape[0], 1), dtype=np.uint64)
    if roots.shape[0] == 0:
        return np.zeros((0, 5), dtype=np.uint64) if bytes_b else out
    rc = lib.orc_per_root(g.nU, g.nV, _p32(uo), _p32(ua), _p32(vo), _p32(va), _p32(roots), roots.shape[0],
                          out.ctypes.data_as(_U64P), nthreads, ob.ctypes.data_as(_U64P), int(min_r), int(min_l),
                          int(bool(prune)))
    if rc:
        raise MemoryError("oracle per-root run failed")
    if bytes_b:
        return np.concatenate([out, ob[:roots.shape[0], None]], axis=1)
    return out


def root_order(g) -> np.ndarray:
    """The top-level pop sequence: non-isolated U vertices by (degree, id)."""
    lib = _load()
    uo = _c32(g.u_off)
    seq = np.zeros(max(g.nU, 1), dtype=np.int32)
    n = ctypes.c_int64(0)
    if lib.orc_root_order(g.nU, _p32(uo), _p32(seq), ctypes.byref(n)):
        raise MemoryError
    return seq[:n.value].copy()


def batch(b, nthreads: int = 1, order=None) -> np.ndarray:
    """Per-graph (count, hash, nodes, bytes) for a packed batch; uint64 array [G, 4]."""
    lib = _load()
    G = b.n_graphs
    out = np.zeros((G, 4), dtype=np.uint64)
    if G == 0:
        return out
    arrs = dict(nU=_c32(b.nU), nV=_c32(b.nV), eo=np.ascontiguousarray(b.edge_off, np.int64),
                us=np.ascontiguousarray(b.u_off_start, np.int64), vs=np.ascontiguousarray(b.v_off_start, np.int64),
                uo=_c32(b.u_off), ua=_c32(b.u_adj), vo=_c32(b.v_off), va=_c32(b.v_adj))
    order = None if order is None else _c32(order)
    rc = lib.orc_batch(G, _p32(arrs["nU"]), _p32(arrs["nV"]), arrs["eo"].ctypes.data_as(_I64P),
                       arrs["us"].ctypes.data_as(_I64P), arrs["vs"].ctypes.data_as(_I64P), _p32(arrs["uo"]),
                       _p32(arrs["ua"]), _p32(arrs["vo"]), _p32(arrs["va"]),
                       None if order is None else _p32(order), out.ctypes.data_as(_U64P), nthreads)
    if rc:
        raise MemoryError("oracle batch run failed")
    return out


def bruteforce(g, records: bool = False):
    """Closure enumeration over all subsets of U (|U| <= 24): ``(count, hash[, records])``."""
    lib = _load()
    if g.nU > 24:
        raise ValueError("brute force needs |U| <= 24")
    uo, ua = _c32(g.u_off), _c32(g.u_adj)
    out = np.zeros(2, dtype=np.uint64)
    rec_p, rec_n = _I32P(), ctypes.c_int64(0)
    rc = lib.orc_bruteforce(g.nU, g.nV, _p32(uo), _p32(ua), out.ctypes.data_as(_U64P),
                            ctypes.byref(rec_p) if records else None, ctypes.byref(rec_n) if records else None)
    if rc:
        raise MemoryError("brute force failed")
    res = (int(out[0]), int(out[1]))
    if records:
        return res + (_records(rec_p, rec_n),)
    return res


def biclique_hash(pairs) -> int:
    """The order-independent digest of a list of (R, L) pairs, via the oracle's SplitMix64."""
    h = 0
    for r, l in pairs:
        s = 0
        for u in r:
            s = (s + sm(2 * u)) & 0xFFFFFFFFFFFFFFFF
        for v in l:
            s = (s + sm(2 * v + 1)) & 0xFFFFFFFFFFFFFFFF
        h = (h + sm(s)) & 0xFFFFFFFFFFFFFFFF
    return h

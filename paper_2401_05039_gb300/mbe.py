"""Thin ctypes binding of the C ABI in include/mbe.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/libmbe.so``; this module
converts numpy arrays (host memory) and torch CUDA tensors (device memory)
to raw pointers and turns status codes into exceptions. There is no CPU
fallback: without the library (or a GPU) the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

MBE_OK = 0
STATUS = {0: "MBE_OK", 1: "MBE_ERR_INVALID_ARG", 2: "MBE_ERR_INVALID_GRAPH", 3: "MBE_ERR_OOM",
          4: "MBE_ERR_ARENA_FULL", 5: "MBE_ERR_OUTPUT_FULL", 6: "MBE_ERR_TIMEOUT", 7: "MBE_ERR_CUDA",
          8: "MBE_ERR_UNSUPPORTED", 9: "MBE_ERR_INTERNAL"}


class MBEError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class Options(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("bitset_max_words", ctypes.c_int32), ("steal", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("emit", ctypes.c_int32), ("watchdog_ms", ctypes.c_int32), ("root_begin", ctypes.c_int32),
                ("root_end", ctypes.c_int32), ("arena_bytes", ctypes.c_int64), ("model", ctypes.c_void_p),
                ("per_root", ctypes.c_void_p), ("exec_order", ctypes.c_void_p), ("n_exec", ctypes.c_int32),
                ("class_params", ctypes.c_void_p), ("layout", ctypes.c_int32), ("min_r", ctypes.c_int32),
                ("min_l", ctypes.c_int32), ("prune", ctypes.c_int32)]


class ClassParams(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("steal", ctypes.c_int32),
                ("valid", ctypes.c_int32), ("layout", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("tuned_ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


N_CLASSES = 8


class Result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("hash", ctypes.c_uint64), ("nodes", ctypes.c_uint64),
                ("bytes_alg", ctypes.c_uint64), ("device_ms", ctypes.c_double), ("prep_ms", ctypes.c_double),
                ("status", ctypes.c_int32), ("n_workers", ctypes.c_int32), ("n_donations", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BicliqueBuffer(ctypes.Structure):
    _fields_ = [("ids", ctypes.c_void_p), ("capacity_ids", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("capacity_bicliques", ctypes.c_int64), ("n_ids_written", ctypes.c_int64),
                ("n_bicliques_written", ctypes.c_int64)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

_SIGNATURES = {
    "mbe_status_string": ([_I32], ctypes.c_char_p),
    "mbe_graph_create": ([_I32, _I32, _I64, _P, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)], _I32),
    "mbe_graph_destroy": ([_P], _I32),
    "mbe_graph_info": ([_P, _P, _P, _P, _P, _P], _I32),
    "mbe_default_options": ([ctypes.POINTER(Options)], _I32),
    "mbe_enumerate": ([_P, ctypes.POINTER(Options), _P, ctypes.POINTER(Result), ctypes.POINTER(BicliqueBuffer)], _I32),
    "mbe_release_workspace": ([], _I32),
    "mbe_debug_trace": ([_P, _I32], _I32),
    "mbe_enumerate_noalloc": ([_I32, _I32, _I64, _P, _P, _P, _P, _P, ctypes.POINTER(Result)], _I32),
    "mbe_copy_bandwidth": ([_I64, _I32, _P, ctypes.POINTER(ctypes.c_double)], _I32),
    "mbe_batch_class": ([_I32, _I32, _I64], _I32),
    "mbe_model_create": ([ctypes.c_uint64, ctypes.POINTER(_P)], _I32),
    "mbe_model_destroy": ([_P], _I32),
    "mbe_model_set_params": ([_P, _P], _I32),
    "mbe_model_get_params": ([_P, _P], _I32),
    "mbe_root_features": ([_P, _P, _P, _P], _I32),
    "mbe_model_predict": ([_P, _P, _I32, _P, _P], _I32),
    "mbe_model_loss_grad": ([_P, _P, _P, _I32, _P, ctypes.POINTER(ctypes.c_float), _P], _I32),
    "mbe_model_train": ([_P, _P, _P, _I32, _I32, _I32, ctypes.c_float, ctypes.c_uint64, _P,
                         ctypes.POINTER(ctypes.c_float)], _I32),
    "mbe_autotune_batch": ([_I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I32, _P, _P], _I32),
    "mbe_enumerate_batch": ([_I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(Options), _P, _P,
                             ctypes.POINTER(Result)], _I32),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmbe.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            # MBE_LIBRARY points the binding at another build of the same sources
            path = os.environ.get("MBE_LIBRARY") or (_build.build() if build_if_missing else _build.LIB)
            if not os.path.exists(path):
                raise ImportError(f"CUDA library not built: {path}")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _check(st: int, what: str):
    if st != MBE_OK:
        raise MBEError(st, what)


def _ptr(x):
    """Raw pointer of a numpy array (host) or a torch tensor (device or host)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def options(**kw) -> Options:
    o = Options()
    _check(load().mbe_default_options(ctypes.byref(o)), "mbe_default_options")
    for k, v in kw.items():
        if k == "class_params" and v is not None and not isinstance(v, int):
            v = ctypes.cast(v, ctypes.c_void_p).value
        elif k == "model" and isinstance(v, Model):
            v = v.handle
        elif k in ("per_root", "exec_order", "model"):
            v = _ptr(v) if not isinstance(v, (int, type(None))) else v
        setattr(o, k, v)
    return o


class Graph:
    """A graph handle: wraps mbe_graph_create / mbe_enumerate / mbe_graph_destroy."""

    def __init__(self, nU, nV, u_off, u_adj, v_off, v_adj, stream=None):
        lib = load()
        device = (not isinstance(u_off, np.ndarray)) and bool(getattr(u_off, "is_cuda", False))
        if isinstance(u_off, np.ndarray):
            u_off, u_adj, v_off, v_adj = (np.ascontiguousarray(a, dtype=np.int32) for a in (u_off, u_adj, v_off, v_adj))
        if device:
            _check_device_graph(int(nU), int(nV), u_off, u_adj, v_off, v_adj)
        elif (int(u_off.shape[0]) != int(nU) + 1 or int(v_off.shape[0]) != int(nV) + 1
              or int(u_adj.shape[0]) != int(v_adj.shape[0])):
            raise MBEError(1, "u_off needs nU + 1 entries, v_off nV + 1, and u_adj / v_adj one per edge")
        self._keep = (u_off, u_adj, v_off, v_adj)
        h = _P()
        nE = int(u_adj.shape[0])
        st = lib.mbe_graph_create(int(nU), int(nV), nE, _ptr(u_off), _ptr(u_adj), _ptr(v_off), _ptr(v_adj),
                                  1 if device else 0, _stream_handle(stream), ctypes.byref(h))
        _check(st, "mbe_graph_create")
        self._h = h
        self.nU, self.nV, self.nE = int(nU), int(nV), nE

    @classmethod
    def from_synth(cls, g, stream=None):
        return cls(g.nU, g.nV, g.u_off, g.u_adj, g.v_off, g.v_adj, stream=stream)

    def info(self):
        vals = [ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()]
        _check(load().mbe_graph_info(self._h, *[ctypes.byref(v) for v in vals]), "mbe_graph_info")
        return dict(zip(("nU", "nV", "nE", "max_deg_u", "max_deg_v"), (v.value for v in vals)))

    def enumerate(self, stream=None, bicliques=None, check=True, **kw) -> Result:
        """Run mbe_enumerate; kw are mbe_options fields. bicliques: BicliqueBuffer or None."""
        o = options(**kw)
        r = Result()
        st = load().mbe_enumerate(self._h, ctypes.byref(o), _stream_handle(stream), ctypes.byref(r),
                                  ctypes.byref(bicliques) if bicliques is not None else None)
        if check:
            _check(st, "mbe_enumerate")
        return r

    def iter_bicliques(self, capacity_ids=1 << 24, capacity_bicliques=1 << 20, pinned_host=True, stream=None,
                       **kw):
        """Every maximal biclique as (R, L) id tuples (each ascending), in bounded memory.

        The roots of the static order are taken in contiguous shards
        (root_begin / root_end); each shard is enumerated into one reused
        buffer of the given capacities, in pinned host memory by default (the
        kernels write it directly), and a shard whose output does not fit is
        halved and run again. kw are further mbe_options fields (layout,
        min_r, min_l, ...). The shards' bicliques are those of the whole graph.
        """
        import torch
        u_off = self._keep[0]
        deg = u_off[1:] - u_off[:-1]
        n_roots = int((deg > 0).sum())
        buf = Bicliques.allocate(capacity_ids, capacity_bicliques, pinned_host=pinned_host)
        stack = [(0, n_roots)]
        while stack:
            b, e = stack.pop()
            if b >= e:
                continue
            r = self.enumerate(stream=stream, bicliques=buf.buf, check=False, emit=1, root_begin=b, root_end=e, **kw)
            if r.status == 5 and e - b > 1:  # MBE_ERR_OUTPUT_FULL: split the shard
                mid = (b + e) // 2
                stack.append((mid, e))
                stack.append((b, mid))
                continue
            _check(r.status, "mbe_enumerate")
            torch.cuda.synchronize()
            yield from buf.records()

    def features(self, stream=None, raw=False):
        """mbe_root_features: float32 [nU, 8] CUDA tensor (and the raw int32 values with raw=True)."""
        import torch
        f = torch.zeros((self.nU, 8), dtype=torch.float32, device="cuda")
        r = torch.zeros((self.nU, 8), dtype=torch.int32, device="cuda") if raw else None
        _check(load().mbe_root_features(self._h, f.data_ptr(), r.data_ptr() if raw else None,
                                        _stream_handle(stream)), "mbe_root_features")
        return (f, r) if raw else f

    def per_root(self, stream=None, **kw):
        """(Result, uint64 numpy [nU, 4]) with the per-root (count, hash, nodes, bytes)."""
        import torch
        buf = torch.zeros((self.nU, 4), dtype=torch.int64, device="cuda")
        r = self.enumerate(stream=stream, per_root=buf, **kw)
        return r, buf.cpu().numpy().view(np.uint64)

    def close(self):
        if getattr(self, "_h", None):
            load().mbe_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def _batch_arrays(b):
    return [np.ascontiguousarray(b.edge_off, np.int64), np.ascontiguousarray(b.nU, np.int32),
            np.ascontiguousarray(b.nV, np.int32), np.ascontiguousarray(b.u_off_start, np.int64),
            np.ascontiguousarray(b.v_off_start, np.int64), np.ascontiguousarray(b.u_off, np.int32),
            np.ascontiguousarray(b.u_adj, np.int32), np.ascontiguousarray(b.v_off, np.int32),
            np.ascontiguousarray(b.v_adj, np.int32)]


def batch_class(nU, nV, nE) -> int:
    return int(load().mbe_batch_class(int(nU), int(nV), int(nE)))


def autotune_batch(b, sample_per_class=64, stream=None):
    """mbe_autotune_batch: returns the per-class parameter table (ClassParams * N_CLASSES)."""
    table = (ClassParams * N_CLASSES)()
    arrs = _batch_arrays(b)
    _check(load().mbe_autotune_batch(int(b.n_graphs), *[a.ctypes.data for a in arrs], int(sample_per_class),
                                     _stream_handle(stream), ctypes.cast(table, _P)), "mbe_autotune_batch")
    return table


def enumerate_batch(b, stream=None, check=True, **kw):
    """mbe_enumerate_batch over a packed batch (host arrays). Returns (list of Result, total Result)."""
    lib = load()
    G = int(b.n_graphs)
    arrs = _batch_arrays(b)
    per = (Result * max(G, 1))()
    tot = Result()
    o = options(**kw)
    st = lib.mbe_enumerate_batch(G, *[a.ctypes.data for a in arrs], ctypes.byref(o), _stream_handle(stream),
                                 ctypes.cast(per, _P), ctypes.byref(tot))
    if check:
        _check(st, "mbe_enumerate_batch")
    return [per[i] for i in range(G)], tot


def copy_bandwidth(nbytes: int, iters: int = 5, stream=None) -> float:
    """Best device copy bandwidth in GB/s (read + write) over `iters` copies of `nbytes`."""
    out = ctypes.c_double()
    _check(load().mbe_copy_bandwidth(int(nbytes), int(iters), _stream_handle(stream), ctypes.byref(out)),
           "mbe_copy_bandwidth")
    return out.value


def _check_device_graph(nU, nV, u_off, u_adj, v_off, v_adj):
    """Shape, dtype and placement of a graph given as device tensors (the library reads raw pointers)."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("u_off", u_off), ("u_adj", u_adj), ("v_off", v_off), ("v_adj", v_adj)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != dev:
            raise MBEError(1, f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != torch.int32 or t.dim() != 1 or not t.is_contiguous():
            raise MBEError(1, f"{name} must be a contiguous 1-D int32 tensor")
    if nU < 0 or nV < 0 or u_off.numel() != nU + 1 or v_off.numel() != nV + 1:
        raise MBEError(1, "u_off needs nU + 1 entries and v_off nV + 1")
    if u_adj.numel() != v_adj.numel():
        raise MBEError(1, "u_adj and v_adj must have the same length (one entry per edge)")


def enumerate_noalloc(nU, nV, u_off, u_adj, v_off, v_adj, stream=None, check=True) -> Result:
    """mbe_enumerate_noalloc on DEVICE arrays (torch CUDA tensors); allocates nothing."""
    _check_device_graph(int(nU), int(nV), u_off, u_adj, v_off, v_adj)
    r = Result()
    st = load().mbe_enumerate_noalloc(int(nU), int(nV), int(u_adj.shape[0]), _ptr(u_off), _ptr(u_adj), _ptr(v_off),
                                      _ptr(v_adj), _stream_handle(stream), ctypes.byref(r))
    if check:
        _check(st, "mbe_enumerate_noalloc")
    return r


class Model:
    """The cost network (mbe_model_*): FP32 master weights, FP16 copy, trained on the GPU."""

    N_PARAMS = 4801

    def __init__(self, seed: int = 0):
        h = _P()
        _check(load().mbe_model_create(ctypes.c_uint64(seed), ctypes.byref(h)), "mbe_model_create")
        self._h = h

    @property
    def handle(self):
        return self._h.value

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.N_PARAMS
        _check(load().mbe_model_set_params(self._h, p.ctypes.data), "mbe_model_set_params")

    def get_params(self):
        p = np.zeros(self.N_PARAMS, dtype=np.float32)
        _check(load().mbe_model_get_params(self._h, p.ctypes.data), "mbe_model_get_params")
        return p

    def predict(self, feat, stream=None):
        import torch
        out = torch.empty(feat.shape[0], dtype=torch.float32, device="cuda")
        _check(load().mbe_model_predict(self._h, feat.data_ptr(), int(feat.shape[0]), out.data_ptr(),
                                        _stream_handle(stream)), "mbe_model_predict")
        return out

    def loss_grad(self, feat, target, stream=None):
        g = np.zeros(self.N_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(load().mbe_model_loss_grad(self._h, feat.data_ptr(), target.data_ptr(), int(feat.shape[0]),
                                          g.ctypes.data, ctypes.byref(loss), _stream_handle(stream)),
               "mbe_model_loss_grad")
        return float(loss.value), g

    def train(self, feat, target, epochs=30, batch=512, lr=3e-3, seed=0, stream=None):
        loss = ctypes.c_float()
        _check(load().mbe_model_train(self._h, feat.data_ptr(), target.data_ptr(), int(feat.shape[0]), int(epochs),
                                      int(batch), ctypes.c_float(lr), ctypes.c_uint64(seed), _stream_handle(stream),
                                      ctypes.byref(loss)), "mbe_model_train")
        return float(loss.value)

    def close(self):
        if getattr(self, "_h", None):
            load().mbe_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def training_set(graphs, stream=None):
    """Features and log1p(subtree nodes) of every non-isolated root of each graph (CUDA tensors).

    The labels are the per-root node counts logged by a plain enumeration of
    the graph; isolated roots are left out.
    """
    import torch
    feats, targets = [], []
    for g in graphs:
        G = Graph.from_synth(g, stream=stream)
        _, pr = G.per_root(stream=stream)
        f = G.features(stream=stream)
        live = torch.from_numpy(np.diff(g.u_off) > 0).cuda()
        feats.append(f[live])
        targets.append(torch.log1p(torch.from_numpy(pr[:, 2].astype(np.float64)).cuda()[live]).float())
        G.close()
    return torch.cat(feats).contiguous(), torch.cat(targets).contiguous()


def release_workspace():
    _check(load().mbe_release_workspace(), "mbe_release_workspace")


@dataclass
class Bicliques:
    """Device buffers for emitted bicliques plus the decoded host view."""

    ids: object
    offsets: object
    buf: BicliqueBuffer

    @classmethod
    def allocate(cls, capacity_ids: int, capacity_bicliques: int, pinned_host: bool = False):
        """Buffers in device memory, or (pinned_host) in pinned host memory that the kernels write directly."""
        import torch
        if pinned_host:
            ids = torch.empty(max(capacity_ids, 1), dtype=torch.int32).pin_memory()
            offs = torch.empty(max(capacity_bicliques, 1), dtype=torch.int64).pin_memory()
        else:
            ids = torch.empty(max(capacity_ids, 1), dtype=torch.int32, device="cuda")
            offs = torch.empty(max(capacity_bicliques, 1), dtype=torch.int64, device="cuda")
        buf = BicliqueBuffer(ids.data_ptr(), capacity_ids, offs.data_ptr(), capacity_bicliques, 0, 0)
        return cls(ids, offs, buf)

    def records(self):
        """The (R, L) id tuples as written (each side already ascending)."""
        n = int(self.buf.n_bicliques_written)
        ids = self.ids.cpu().numpy()
        for o in self.offsets[:n].cpu().numpy().tolist():
            nr, nl = int(ids[o]), int(ids[o + 1])
            yield tuple(ids[o + 2:o + 2 + nr].tolist()), tuple(ids[o + 2 + nr:o + 2 + nr + nl].tolist())

    def decode(self):
        """List of (R, L) sorted tuples for the bicliques written."""
        n = int(self.buf.n_bicliques_written)
        ids = self.ids.cpu().numpy()
        offs = self.offsets[:n].cpu().numpy()
        out = []
        for o in offs.tolist():
            nr, nl = int(ids[o]), int(ids[o + 1])
            r = tuple(sorted(ids[o + 2:o + 2 + nr].tolist()))
            l = tuple(sorted(ids[o + 2 + nr:o + 2 + nr + nl].tolist()))
            out.append((r, l))
        return out


# ------------------------------------------------------------ several ranks
# Roots are independent units: a graph's execution order can be split into
# contiguous shards (mbe_options.root_begin / root_end), one per rank, and the
# shard results add up (count, nodes, bytes as integers, the hash mod 2^64).

def shard_bounds(n: int, rank: int, world: int):
    """[begin, end) of rank's contiguous share of n roots (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    q, r = divmod(n, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def allreduce_totals(totals, group=None):
    """Sum (count, hash, nodes, bytes) over the ranks of a torch.distributed group.

    The values are split into 16-bit limbs in int64 tensors, so the sums are
    exact for any number of ranks that fits in 2^47, on any backend (gloo on
    the CPU, NCCL on GPUs); the hash is returned mod 2^64.
    """
    import torch
    import torch.distributed as dist
    vals = [int(v) & 0xFFFFFFFFFFFFFFFF for v in totals]
    limbs = torch.tensor([[(v >> (16 * k)) & 0xFFFF for k in range(4)] for v in vals], dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        limbs = limbs.cuda()
    dist.all_reduce(limbs, op=dist.ReduceOp.SUM, group=group)
    out = [sum(int(x) << (16 * k) for k, x in enumerate(row)) for row in limbs.cpu().tolist()]
    out[1] &= 0xFFFFFFFFFFFFFFFF
    return tuple(out)


def lpt_shards(cost, world: int):
    """Roots assigned to `world` ranks, longest processing time first.

    cost[u] is the expected cost of root u (a prediction of the cost network
    or a static proxy); roots with cost <= 0 (isolated vertices) are left
    out. Roots are taken in descending cost and each goes to the rank with
    the least load so far, so the largest load is at most 4/3 of the best
    possible. Returns one int32 array of root ids per rank, in descending
    cost (the order in which that rank should run them).
    """
    import heapq
    if world < 1:
        raise ValueError("need world >= 1")
    cost = np.asarray(cost, dtype=np.float64)
    ids = np.nonzero(cost > 0)[0]
    order = ids[np.argsort(-cost[ids], kind="stable")]
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for u in order.tolist():
        load, r = heapq.heappop(heap)
        out[r].append(u)
        heapq.heappush(heap, (load + float(cost[u]), r))
    return [np.asarray(o, dtype=np.int32) for o in out]


def static_root_cost(raw_features):
    """Static cost proxy of every root from mbe_root_features' raw values.

    The number of (neighbour, second neighbour) pairs the root's setup reads
    (sum of the degrees of N(r)) times its candidate count |N2(r)|; zero for
    isolated roots.
    """
    raw = np.asarray(raw_features, dtype=np.float64)
    return raw[:, 5] * np.maximum(raw[:, 1], 1.0) * (raw[:, 0] > 0)


def sharded_enumerate(graph, rank: int, world: int, n_roots: int = 0, group=None, cost=None, **kw):
    """Rank's shard of the graph's roots, enumerated on this rank's GPU and summed over the group.

    Without `cost`: the contiguous equal-count share [begin, end) of the
    static execution order (n_roots = its length). With `cost` (per root id):
    the rank's LPT share (lpt_shards), run as an explicit execution order.
    """
    if cost is None:
        b, e = shard_bounds(n_roots, rank, world)
        r = graph.enumerate(root_begin=b, root_end=e, **kw)
    else:
        import torch
        mine = lpt_shards(cost, world)[rank]
        order = torch.from_numpy(mine).cuda()
        r = graph.enumerate(exec_order=order, n_exec=int(mine.shape[0]), **kw)
    return allreduce_totals((r.count, r.hash, r.nodes, r.bytes_alg), group)

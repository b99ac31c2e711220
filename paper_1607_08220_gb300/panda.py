"""Thin Python binding of the C ABI in include/panda.h (argument marshalling only).

Every step of the build and the query runs in the CUDA library
(``_lib/libpanda.so``); this module only passes pointers, sizes and streams.
PyTorch provides device memory and streams.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise :class:`PandaError`.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpanda.so")

ORDER = {"none": 0, "morton": 1, "leaf": 2}
TRAVERSAL = {"auto": 0, "packet": 1, "per_query": 2}
STATUS_TIMEOUT = 6
STATUS_NAMES = {0: "PANDA_OK", 1: "PANDA_ERR_INVALID_ARGUMENT", 2: "PANDA_ERR_NONFINITE_INPUT",
                3: "PANDA_ERR_UNSUPPORTED", 4: "PANDA_ERR_OUT_OF_MEMORY", 5: "PANDA_ERR_CUDA",
                6: "PANDA_ERR_TIMEOUT", 7: "PANDA_ERR_QUEUE_FULL", 8: "PANDA_ERR_DEPTH"}

# Every symbol include/panda.h declares, with its ctypes signature.
_P, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "panda_build": ([_P, _I64, _I32, _I32, ctypes.POINTER(_P)], ctypes.c_int),
    "panda_build_async": ([_P, _I64, _I32, _I32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "panda_build_host": ([_P, _I64, _I32, _I32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "panda_knn": ([_P, _P, _I64, _I32, _P, _P], ctypes.c_int),
    "panda_knn_async": ([_P, _P, _I64, _I32, _P, _P, _P, _P], ctypes.c_int),
    "panda_knn_host": ([_P, _P, _I64, _I32, _P, _P, _P, _P], ctypes.c_int),
    "panda_knn_self": ([_P, _I32, _P, _P], ctypes.c_int),
    "panda_knn_vote": ([_P, _I64, _I32, _P, _I64, _P, _P], ctypes.c_int),
    "panda_refit": ([_P, _P, _P], ctypes.c_int),
    "panda_tree_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "panda_tree_load": ([ctypes.c_char_p, _P], ctypes.c_int),
    "panda_knn_mean": ([_P, _I64, _I32, _P, _I64, _P, _P], ctypes.c_int),
    "panda_knn_self_async": ([_P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "panda_knn_self_host": ([_P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "panda_knn_self_host_async": ([_P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "panda_free_async": ([_P, _P], None),
    "panda_knn_visits": ([_P, _P, _I64, _I32, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "panda_knn_noalloc": ([_P, _P, _I64, _I32, _P, _P, _P], ctypes.c_int),
    "panda_batch_create": ([_P, _I32, _I32, _I32, ctypes.POINTER(_P)], ctypes.c_int),
    "panda_batch_buffers": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "panda_batch_offsets": ([_P, _P, _P, _P], ctypes.c_int),
    "panda_batch_run": ([_P, _P], ctypes.c_int),
    "panda_batch_status": ([_P, _P], ctypes.c_int),
    "panda_batch_info": ([_P, _P, _P], ctypes.c_int),
    "panda_batch_free": ([_P], None),
    "panda_server_create": ([_I64, _I64, ctypes.POINTER(_P)], ctypes.c_int),
    "panda_server_add_tree": ([_P, _P, _I64, _I32, _I32, _P], ctypes.c_int),
    "panda_server_submit": ([_P, _I32, _P, _I64, _I32, _P, _P, _P], ctypes.c_int),
    "panda_server_poll": ([_P, _I64, _P], ctypes.c_int),
    "panda_server_set_queue_limit": ([_P, _I64], ctypes.c_int),
    "panda_server_admission": ([_P, _P, _P, _P], ctypes.c_int),
    "panda_server_wait": ([_P, _I64, _I64], ctypes.c_int),
    "panda_server_request_info": ([_P, _I64, _P, _P, _P], ctypes.c_int),
    "panda_server_now_ns": ([_P], _I64),
    "panda_server_stats": ([_P, _P, _P, _P, _P], ctypes.c_int),
    "panda_server_destroy": ([_P], None),
    "panda_tune": ([_P, _I64, _I32, _P, _I64, _I64, _I32, _P, _P], ctypes.c_int),
    "panda_tune_lookup": ([_I32, _I64, _I32, _I64, _P], ctypes.c_int),
    "panda_batch_set_query_params": ([_P, _P], ctypes.c_int),
    "panda_free": ([_P], None),
    "panda_tree_get_info": ([_P, _P], ctypes.c_int),
    "panda_tree_copy": ([_P, _P, _P], ctypes.c_int),
    "panda_set_phase_timing": ([_I32], None),
    "panda_phase_times": ([_P, _P, _P, _I32], _I32),
    "panda_kernel_launches": ([], _I64),
    "panda_debug_fail_alloc": ([_I64], ctypes.c_int),
    "panda_debug_pool_used": ([_P], ctypes.c_int),
    "panda_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "panda_last_error": ([], ctypes.c_char_p),
    "panda_version": ([], ctypes.c_char_p),
}


class PandaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class QueryParams(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("transpose_max", ctypes.c_int32), ("traversal", ctypes.c_int32),
                ("bounded", ctypes.c_int32), ("max_d2", ctypes.c_float), ("reserved", ctypes.c_int32)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("bucket", ctypes.c_int32),
                ("num_nodes", ctypes.c_int64), ("num_leaves", ctypes.c_int64),
                ("depth", ctypes.c_int32), ("node_floats", ctypes.c_int32),
                ("point_floats", ctypes.c_int32), ("subtree_threshold", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("node_slots", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libpanda.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise PandaError(5, f"CUDA library not built: {p} (run paper_1607_08220_gb300.build_ext)")
        L = ctypes.CDLL(p)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(st: int):
    if st != 0:
        msg = _lib.panda_last_error().decode(errors="replace")
        raise PandaError(st, msg)


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Tree:
    """A kd-tree resident in device memory (owns a C handle)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = TreeInfo()
        _check(_lib.panda_tree_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in TreeInfo._fields_}

    def free(self, stream=None):
        """Release the device memory (stream given: in that stream's order)."""
        if self._h:
            if stream is None:
                _lib.panda_free(self._h)
            else:
                _lib.panda_free_async(self._h, _stream_ptr(stream))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def raw(self):
        """(nodes [num_nodes][node_floats] float32, points [n][point_floats] float32) on the host."""
        inf = self.info()
        nodes = np.empty((inf["node_slots"], inf["node_floats"]), np.float32)
        pts = np.empty((inf["n"], inf["point_floats"]), np.float32)
        _check(_lib.panda_tree_copy(self._h, nodes.ctypes.data_as(ctypes.c_void_p),
                                    pts.ctypes.data_as(ctypes.c_void_p)))
        return nodes, pts

    def export(self) -> dict:
        """Canonical preorder form (the same layout the oracle exports)."""
        inf = self.info()
        d = inf["d"]
        nodes, pts = self.raw()
        return canonical_from_raw(nodes, pts, d)


def padded_dim(d: int) -> int:
    if d <= 2:
        return 2
    if d <= 4:
        return d
    if d <= 8:
        return 8
    if d <= 10:
        return 10
    return 16


def canonical_from_raw(nodes: np.ndarray, pts: np.ndarray, d: int) -> dict:
    """Walk the node table from the root in preorder; children of an inner node
    are (a, a+1); a leaf covers packed points a .. a+b-1."""
    dp = padded_dim(d)
    hdr = nodes[:, :4].view(np.int32)
    a_col, b_col, meta = hdr[:, 0], hdr[:, 1], hdr[:, 3].view(np.uint32)
    split_col = nodes[:, 2]
    order, depth, parent_slot = [], [], []
    stack = [(0, 0)]
    while stack:
        i, dep = stack.pop()
        order.append(i)
        depth.append(dep)
        if not meta[i] & 0x80000000:
            c = int(a_col[i])
            stack.append((c + 1, dep + 1))
            stack.append((c, dep + 1))
    order = np.asarray(order, np.int64)
    pos = np.full(nodes.shape[0], -1, np.int64)
    pos[order] = np.arange(order.size)
    m = meta[order]
    leaf = (m & 0x80000000) != 0
    left = np.where(leaf, -1, pos[np.where(leaf, 0, a_col[order])])
    right = np.where(leaf, -1, pos[np.where(leaf, 0, a_col[order] + 1)])
    start = np.zeros(order.size, np.int64)
    count = np.zeros(order.size, np.int64)
    start[leaf] = a_col[order][leaf]
    count[leaf] = b_col[order][leaf]
    for j in range(order.size - 1, -1, -1):   # children follow their parent in preorder
        if not leaf[j]:
            start[j] = start[left[j]]
            count[j] = count[left[j]] + count[right[j]]
    ids = pts[:, dp].copy().view(np.int32)
    return dict(leaf=leaf, index_split=((m & 0x40000000) != 0) & ~leaf,
                dim=(m & 31).astype(np.int32), depth=np.asarray(depth, np.int32),
                split=split_col[order].copy(), start=start, count=count, left=left, right=right,
                lo=nodes[order, 4:4 + d].copy(), hi=nodes[order, 4 + dp:4 + dp + d].copy(),
                perm=ids)


class TuneResult(ctypes.Structure):
    _fields_ = [("bucket", ctypes.c_int32), ("order", ctypes.c_int32), ("transpose_max", ctypes.c_int32),
                ("traversal", ctypes.c_int32), ("build_ms", ctypes.c_float), ("query_ms", ctypes.c_float),
                ("score_ms", ctypes.c_float), ("reserved2", ctypes.c_float)]


ORDER_NAMES = {v: k for k, v in ORDER.items()}


def _params(order="leaf", transpose_max=0, traversal="auto", max_d2=None) -> "QueryParams":
    """Query parameters; max_d2 (squared search radius, Algorithm 1's r^2) bounds
    the neighbours to d2 <= max_d2 when given."""
    o = ORDER[order] if isinstance(order, str) else int(order)
    if max_d2 is None:
        return QueryParams(o, int(transpose_max), TRAVERSAL[traversal], 0, 0.0, 0)
    return QueryParams(o, int(transpose_max), TRAVERSAL[traversal], 1, float(max_d2), 0)
TRAVERSAL_NAMES = {v: k for k, v in TRAVERSAL.items()}


def tune(points, queries_sample, k: int, m_total: int, stream=None) -> dict:
    """panda_tune: pick bucket size, query order and scan shape by timing them."""
    p = _as_device_points(points, "points")
    q = _as_device_points(queries_sample, "queries")
    r = TuneResult()
    _check(load().panda_tune(ctypes.c_void_p(p.data_ptr()), p.shape[0], p.shape[1], ctypes.c_void_p(q.data_ptr()),
                             q.shape[0], int(m_total), int(k), _stream_ptr(stream), ctypes.byref(r)))
    return dict(bucket=r.bucket, order=ORDER_NAMES[r.order], transpose_max=r.transpose_max,
                traversal=TRAVERSAL_NAMES[r.traversal], build_ms=r.build_ms, query_ms=r.query_ms,
                score_ms=r.score_ms)


def tune_lookup(d: int, n: int, k: int, m_total: int):
    r = TuneResult()
    st = load().panda_tune_lookup(int(d), int(n), int(k), int(m_total), ctypes.byref(r))
    if st != 0:
        return None
    return dict(bucket=r.bucket, order=ORDER_NAMES[r.order], transpose_max=r.transpose_max,
                traversal=TRAVERSAL_NAMES[r.traversal], build_ms=r.build_ms, query_ms=r.query_ms,
                score_ms=r.score_ms)


class SetDesc(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_queries", ctypes.c_int64), ("k", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class _DeviceArray:
    """Zero-copy view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


class Batch:
    """Batched form: many independent point sets built and queried in one graph launch."""

    def __init__(self, n_points, n_queries, ks, d: int, bucket: int = 32):
        torch = _torch()
        L = load()
        ns = len(n_points)
        descs = (SetDesc * ns)(*[SetDesc(int(a), int(b), int(c), 0) for a, b, c in zip(n_points, n_queries, ks)])
        h = ctypes.c_void_p()
        _check(L.panda_batch_create(descs, ns, int(d), int(bucket), ctypes.byref(h)))
        self._h = h
        self.nsets, self.d = ns, d
        self.ks = [int(k) for k in ks]
        po = (ctypes.c_int64 * (ns + 1))()
        qo = (ctypes.c_int64 * (ns + 1))()
        oo = (ctypes.c_int64 * (ns + 1))()
        _check(L.panda_batch_offsets(h, po, qo, oo))
        self.point_off, self.query_off, self.out_off = list(po), list(qo), list(oo)
        pp, qp, ip, dp = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(L.panda_batch_buffers(h, ctypes.byref(pp), ctypes.byref(qp), ctypes.byref(ip), ctypes.byref(dp)))
        dev = torch.device("cuda", torch.cuda.current_device())
        self.points = torch.as_tensor(_DeviceArray(pp.value, (self.point_off[-1], d), "<f4"), device=dev)
        self.queries = torch.as_tensor(_DeviceArray(qp.value, (max(self.query_off[-1], 1), d), "<f4"),
                                       device=dev)[:self.query_off[-1]]
        self.ids = torch.as_tensor(_DeviceArray(ip.value, (max(self.out_off[-1], 1),), "<i4"),
                                   device=dev)[:self.out_off[-1]]
        self.d2 = torch.as_tensor(_DeviceArray(dp.value, (max(self.out_off[-1], 1),), "<f4"),
                                  device=dev)[:self.out_off[-1]]

    def set_query_params(self, transpose_max: int = 0, traversal: str = "auto"):
        prm = QueryParams(ORDER["leaf"], int(transpose_max), TRAVERSAL[traversal], 0)
        _check(load().panda_batch_set_query_params(self._h, ctypes.byref(prm)))

    def run(self, stream=None):
        _check(load().panda_batch_run(self._h, _stream_ptr(stream)))

    def status(self, stream=None):
        _check(load().panda_batch_status(self._h, _stream_ptr(stream)))

    def result(self, s: int):
        """(ids, d2) of set s as [n_queries][k] views of the output buffers."""
        a, b = self.out_off[s], self.out_off[s + 1]
        k = self.ks[s]
        return self.ids[a:b].view(-1, k), self.d2[a:b].view(-1, k)

    def info(self):
        inf = TreeInfo()
        kr = ctypes.c_int64()
        _check(load().panda_batch_info(self._h, ctypes.byref(inf), ctypes.byref(kr)))
        out = {f: getattr(inf, f) for f, _ in TreeInfo._fields_}
        out["kernels_per_run"] = kr.value
        return out

    def free(self):
        if getattr(self, "_h", None):
            load().panda_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Served form: resident trees and continuous batching of KNN requests."""

    def __init__(self, mem_budget_bytes: int = 0, max_batch_queries: int = 1 << 22):
        h = ctypes.c_void_p()
        _check(load().panda_server_create(int(mem_budget_bytes), int(max_batch_queries), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def add_tree(self, points, bucket: int = 32) -> int:
        p = _as_device_points(points, "points")
        tid = ctypes.c_int32()
        _check(load().panda_server_add_tree(self._h, ctypes.c_void_p(p.data_ptr()), p.shape[0], p.shape[1],
                                            int(bucket), ctypes.byref(tid)))
        return tid.value

    def submit(self, tree_id: int, queries, k: int, out) -> int:
        """Queue a request; `out` = (ids int32 [m][k], d2 float32 [m][k]) CUDA tensors."""
        q = _as_device_points(queries, "queries")
        ids, d2 = out
        rid = ctypes.c_int64()
        _check(load().panda_server_submit(self._h, int(tree_id), ctypes.c_void_p(q.data_ptr()), q.shape[0],
                                          int(k), ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                                          ctypes.byref(rid)))
        self._keep[rid.value] = (q, ids, d2)
        return rid.value

    def poll(self, rid: int) -> bool:
        done = ctypes.c_int32()
        _check(load().panda_server_poll(self._h, int(rid), ctypes.byref(done)))
        return bool(done.value)

    def wait(self, rid: int, timeout_s: float = 60.0):
        st = load().panda_server_wait(self._h, int(rid), int(timeout_s * 1e6))
        if st != STATUS_TIMEOUT:          # finished (well or not): its buffers are free
            self._keep.pop(rid, None)
        _check(st)

    def times(self, rid: int):
        """(submit ns, done ns, batch id) on the server's clock."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().panda_server_request_info(self._h, int(rid), ctypes.byref(a), ctypes.byref(b),
                                                ctypes.byref(c)))
        return a.value, b.value, c.value

    def now_ns(self) -> int:
        return int(load().panda_server_now_ns(self._h))

    def stats(self) -> dict:
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().panda_server_stats(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(["batches", "requests", "pending", "bytes_used"], [x.value for x in v]))

    def set_queue_limit(self, max_pending_queries: int):
        """Cap the queries waiting to be batched (0: no cap); submit beyond it
        raises PANDA_ERR_QUEUE_FULL."""
        _check(load().panda_server_set_queue_limit(self._h, int(max_pending_queries)))

    def admission(self) -> dict:
        """Scratch bytes reserved by the batches in flight, requests that waited
        for memory so far, queries waiting now."""
        v = [ctypes.c_int64() for _ in range(3)]
        _check(load().panda_server_admission(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(["scratch_reserved", "deferred_requests", "pending_queries"], [x.value for x in v]))

    def close(self):
        if getattr(self, "_h", None):
            load().panda_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as_device_points(x, what: str):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise PandaError(1, f"{what} must be a CUDA tensor")
    if x.dtype != torch.float32 or x.dim() != 2:
        raise PandaError(1, f"{what} must be float32 [rows][d]")
    return x.contiguous()


def build(points, bucket: int = 32, stream=None, sync: bool = True) -> Tree:
    """kd-tree over a CUDA float32 tensor [n][d] (Sec. III-A)."""
    L = load()
    pts = _as_device_points(points, "points")
    h = ctypes.c_void_p()
    _check(L.panda_build_async(ctypes.c_void_p(pts.data_ptr()), pts.shape[0], pts.shape[1], int(bucket),
                               _stream_ptr(stream), ctypes.byref(h)))
    t = Tree(h)
    t._keep = pts if not sync else None
    if sync:
        (stream or _torch().cuda.current_stream()).synchronize()
    return t


def knn(tree: Tree, queries, k: int, order: str = "leaf", stream=None, out=None, transpose_max: int = 0,
        traversal: str = "auto", max_d2=None):
    """Exact KNN (Algorithm 1, corrected) of every query row; enqueued on `stream`.

    Returns (ids int32 [m][k], d2 float32 [m][k]) CUDA tensors."""
    torch = _torch()
    L = load()
    q = _as_device_points(queries, "queries")
    m = q.shape[0]
    if out is None:
        ids = torch.empty((m, k), dtype=torch.int32, device=q.device)
        d2 = torch.empty((m, k), dtype=torch.float32, device=q.device)
    else:
        ids, d2 = out
    prm = _params(order, transpose_max, traversal, max_d2)
    _check(L.panda_knn_async(tree.handle, ctypes.c_void_p(q.data_ptr()), m, int(k),
                             ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                             ctypes.byref(prm), _stream_ptr(stream)))
    return ids, d2


def knn_self(tree: Tree, k: int, stream=None, out=None, transpose_max: int = 0, traversal: str = "auto",
             max_d2=None):
    """All-points KNN: every point of the tree is a query (row i = input point i).

    Enqueued on `stream`; returns (ids int32 [n][k], d2 float32 [n][k]) CUDA tensors."""
    torch = _torch()
    L = load()
    n = tree.info()["n"]
    if out is None:
        ids = torch.empty((n, k), dtype=torch.int32, device="cuda")
        d2 = torch.empty((n, k), dtype=torch.float32, device="cuda")
    else:
        ids, d2 = out
    prm = _params("leaf", transpose_max, traversal, max_d2)
    _check(L.panda_knn_self_async(tree.handle, int(k), ctypes.c_void_p(ids.data_ptr()),
                                  ctypes.c_void_p(d2.data_ptr()), ctypes.byref(prm), _stream_ptr(stream)))
    return ids, d2


def knn_self_sync(tree: Tree, k: int):
    """panda_knn_self: blocking all-points query on the legacy stream."""
    torch = _torch()
    L = load()
    n = tree.info()["n"]
    ids = torch.empty((n, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((n, k), dtype=torch.float32, device="cuda")
    torch.cuda.current_stream().synchronize()
    _check(L.panda_knn_self(tree.handle, int(k), ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr())))
    return ids, d2


def knn_self_host(tree: Tree, k: int, stream=None, out: tuple | None = None, max_d2=None, wait: bool = True):
    """panda_knn_self_host: all-points query into host outputs (copy out inside
    the call).  wait=False: panda_knn_self_host_async -- the copy is only
    queued on `stream` (pass pinned outputs and synchronise the stream)."""
    L = load()
    n = tree.info()["n"]
    if out is None:
        ids = np.empty((n, k), np.int32)
        d2 = np.empty((n, k), np.float32)
    else:
        ids, d2 = out
    prm = _params("leaf", 0, "auto", max_d2)
    fn = L.panda_knn_self_host if wait else L.panda_knn_self_host_async
    _check(fn(tree.handle, int(k), ids.ctypes.data_as(ctypes.c_void_p), d2.ctypes.data_as(ctypes.c_void_p),
              ctypes.byref(prm), _stream_ptr(stream)))
    return ids, d2


def save(tree: Tree, path: str):
    """Write the tree to a file (panda_tree_save)."""
    _check(load().panda_tree_save(tree.handle, os.fsencode(path)))


def load_tree(path: str) -> Tree:
    """Read a saved tree onto the current device (panda_tree_load)."""
    h = ctypes.c_void_p()
    _check(load().panda_tree_load(os.fsencode(path), ctypes.byref(h)))
    return Tree(h)


def refit(tree: Tree, points, stream=None):
    """Move the tree's points to new coordinates (CUDA float32 [n][d], original
    id order) and make every box tight again; the structure is kept."""
    L = load()
    pts = _as_device_points(points, "points")
    _check(L.panda_refit(tree.handle, ctypes.c_void_p(pts.data_ptr()), _stream_ptr(stream)))


def knn_vote(ids, labels, stream=None, out=None):
    """Majority label of each row of a KNN result (Sec. I): ids int32 [m][k] and
    labels int32 [n] CUDA tensors; returns int32 [m] (-1: no valid neighbour)."""
    torch = _torch()
    L = load()
    m, k = ids.shape
    if out is None:
        out = torch.empty(m, dtype=torch.int32, device=ids.device)
    _check(L.panda_knn_vote(ctypes.c_void_p(ids.data_ptr()), m, k, ctypes.c_void_p(labels.data_ptr()),
                            labels.shape[0], ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def knn_mean(ids, values, stream=None, out=None):
    """Mean of the neighbours' values (FP32, rank order) of each row of a KNN
    result (Sec. I regression); returns float32 [m] (NaN: no valid neighbour)."""
    torch = _torch()
    L = load()
    m, k = ids.shape
    if out is None:
        out = torch.empty(m, dtype=torch.float32, device=ids.device)
    _check(L.panda_knn_mean(ctypes.c_void_p(ids.data_ptr()), m, k, ctypes.c_void_p(values.data_ptr()),
                            values.shape[0], ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def knn_visits(tree: Tree, queries, k: int, order: str = "leaf", stream=None, transpose_max: int = 0):
    """KNN plus per-query work counts [m][2] (nodes needed, bucket points scanned)
    and the traversal's event counters (dict).  queries=None: the all-points query."""
    torch = _torch()
    L = load()
    if queries is None:
        q, m, qp = None, tree.info()["n"], None
    else:
        q = _as_device_points(queries, "queries")
        m, qp = q.shape[0], q.data_ptr()
    ids = torch.empty((m, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((m, k), dtype=torch.float32, device="cuda")
    vis = torch.zeros((m, 2), dtype=torch.int32, device="cuda")
    stats = torch.zeros(12, dtype=torch.int64, device="cuda")
    prm = QueryParams(ORDER[order], int(transpose_max), 0, 0)
    _check(L.panda_knn_visits(tree.handle, ctypes.c_void_p(qp), m, int(k),
                              ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                              ctypes.c_void_p(vis.data_ptr()), ctypes.c_void_p(stats.data_ptr()),
                              ctypes.byref(prm), _stream_ptr(stream)))
    names = ["warps", "inner_nodes", "bucket_chunks", "lanes_query_chunks", "transposed_broadcasts",
             "insert_rounds", "candidates", "insertions", "pruned_pops", "transposed_insert_rounds",
             "transposed_candidates", "transposed_insertions"]
    return ids, d2, vis, dict(zip(names, stats.cpu().tolist()))


def knn_noalloc(tree: Tree, queries, k: int, out, stream=None):
    """panda_knn_noalloc: the query without any device allocation inside the call.

    For callers that cannot allocate while they query; `out` = (ids, d2) CUDA
    tensors the caller allocated.  At most 2^20 queries per call; calls that
    overlap on the GPU share one scratch array and must be serialised."""
    L = load()
    q = _as_device_points(queries, "queries")
    ids, d2 = out
    _check(L.panda_knn_noalloc(tree.handle, ctypes.c_void_p(q.data_ptr()), q.shape[0], int(k),
                               ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                               _stream_ptr(stream)))
    return ids, d2


def knn_sync(tree: Tree, queries, k: int):
    """panda_knn: blocking query on the legacy stream; checks query finiteness."""
    torch = _torch()
    L = load()
    q = _as_device_points(queries, "queries")
    m = q.shape[0]
    ids = torch.empty((m, k), dtype=torch.int32, device=q.device)
    d2 = torch.empty((m, k), dtype=torch.float32, device=q.device)
    torch.cuda.current_stream().synchronize()
    _check(L.panda_knn(tree.handle, ctypes.c_void_p(q.data_ptr()), m, int(k),
                       ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr())))
    return ids, d2


def build_host(points: np.ndarray, bucket: int = 32, stream=None) -> Tree:
    """panda_build_host: host points; the copy to the device is inside the call."""
    L = load()
    p = np.ascontiguousarray(points, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(L.panda_build_host(p.ctypes.data_as(ctypes.c_void_p), p.shape[0], p.shape[1], int(bucket),
                              _stream_ptr(stream), ctypes.byref(h)))
    return Tree(h)


def knn_host(tree: Tree, queries: np.ndarray, k: int, order: str = "leaf", stream=None,
             out: tuple | None = None, max_d2=None):
    """panda_knn_host: host queries and outputs; copies in and out inside the call."""
    L = load()
    q = np.ascontiguousarray(queries, dtype=np.float32)
    m = q.shape[0]
    if out is None:
        ids = np.empty((m, k), np.int32)
        d2 = np.empty((m, k), np.float32)
    else:
        ids, d2 = out
    prm = _params(order, 0, "auto", max_d2)
    _check(L.panda_knn_host(tree.handle, q.ctypes.data_as(ctypes.c_void_p), m, int(k),
                            ids.ctypes.data_as(ctypes.c_void_p), d2.ctypes.data_as(ctypes.c_void_p),
                            ctypes.byref(prm), _stream_ptr(stream)))
    return ids, d2


def set_phase_timing(on, traversal_only: bool = False):
    """Per-phase CUDA-event timing of the following calls: every phase, or
    (traversal_only) only the traversal, leaving the other kernels unseparated."""
    load().panda_set_phase_timing((2 if traversal_only else 1) if on else 0)


def phase_times() -> list[tuple[str, float, int]]:
    L = load()
    cap = 64
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_float * cap)()
    ln = (ctypes.c_int32 * cap)()
    n = L.panda_phase_times(names, ms, ln, cap)
    return [(names[i].decode(), float(ms[i]), int(ln[i])) for i in range(min(n, cap))]


def kernel_launches() -> int:
    return int(load().panda_kernel_launches())


def debug_fail_alloc(after: int) -> None:
    """Fault injection for tests: after `after` more device workspace
    allocations succeed, the next fails as out of memory (then injection is
    off again); a negative value turns it off."""
    _check(load().panda_debug_fail_alloc(int(after)))


def debug_pool_used() -> int:
    """Bytes the library holds in the stream-ordered pool right now: its own
    count of live trees, forests and call workspace (not what the pool caches,
    nor anyone else's allocations)."""
    v = ctypes.c_int64(0)
    _check(load().panda_debug_pool_used(ctypes.byref(v)))
    return int(v.value)


def version() -> str:
    return load().panda_version().decode()

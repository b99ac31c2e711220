"""Plain CPU oracle for PANDA's kd-tree build and exact KNN (arXiv 1607.08220).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The oracle is C compiled
with ``-O2 -ffp-contract=off`` (no FMA, IEEE round-to-nearest, denormals kept)
and shares no code with the CUDA path.

Functions (each follows the passage cited in ``panda_oracle.c``):

* :func:`build` -- kd-tree construction, Sec. III-A steps ii-iv and Sec. III-A1
  (max-variance split dimension over a 1024-point sample, sampled-histogram
  split value closest to 50%, bucket size B).
* :func:`knn` -- Algorithm 1 (Sec. III-B/C) with the pruning bound, radius
  update and tie handling corrected.
* :func:`brute_knn` -- the plain definition: exhaustive search ordered by
  (FP32 squared distance, point index).

Parity of the traversal work counts (``visits``) is unpinned: the paper prints
no counts, so they serve as diagnostics only.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "panda_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
          "-shared", "-fPIC", "-Wall"]

_lib = None
_lock = threading.Lock()

STATUS = {0: "ok", 1: "invalid argument", 2: "non-finite input", 3: "unsupported",
          4: "out of memory", 5: "depth limit exceeded"}


class OracleError(RuntimeError):
    pass


def lib_path() -> str:
    with open(_SRC, "rb") as f:
        h = hashlib.sha1(f.read() + " ".join(CFLAGS).encode()).hexdigest()[:12]
    return os.path.join(_BUILD_DIR, f"libpanda_oracle_{h}.so")


def compile_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (seconds); returns the shared-library path."""
    path = lib_path()
    if force or not os.path.exists(path):
        os.makedirs(_BUILD_DIR, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, path)
    return path


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = _bind(ctypes.CDLL(compile_oracle()))
        return _lib


def compile_variant(source: str, tag: str):
    """Compile `source` (a modified copy of panda_oracle.c) with the oracle's
    flags and return the loaded library.  For tests that plant a mistake in
    the oracle and check that a pin catches it; the oracle itself is never
    modified."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    h = hashlib.sha1(source.encode() + " ".join(CFLAGS).encode()).hexdigest()[:12]
    path = os.path.join(_BUILD_DIR, f"libpanda_oracle_variant_{tag}_{h}.so")
    if not os.path.exists(path):
        src = path[:-3] + ".c"
        with open(src, "w") as f:
            f.write(source)
        tmp = path + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
        os.replace(tmp, path)
    return _bind(ctypes.CDLL(path))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(L):
    """Declare the C signatures on a loaded oracle library."""
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    L.or_build.argtypes = [P, i64, i32, i32, ctypes.POINTER(P)]
    L.or_build.restype = ctypes.c_int
    L.or_free.argtypes = [P]
    L.or_free.restype = None
    L.or_tree_num_nodes.argtypes = [P]
    L.or_tree_num_nodes.restype = i64
    L.or_tree_depth.argtypes = [P]
    L.or_tree_depth.restype = i32
    L.or_tree_export.argtypes = [P, P, P, P, P, P, P]
    L.or_tree_export.restype = None
    L.or_knn.argtypes = [P, P, i64, i32, P, P, P, i32]
    L.or_knn.restype = ctypes.c_int
    L.or_knn_r.argtypes = [P, P, i64, i32, ctypes.c_float, P, P, P, i32]
    L.or_knn_r.restype = ctypes.c_int
    L.or_brute_knn.argtypes = [P, i64, i32, P, i64, i32, P, P, i32]
    L.or_brute_knn.restype = ctypes.c_int
    L.or_brute_knn_r.argtypes = [P, i64, i32, P, i64, i32, ctypes.c_float, P, P, i32]
    L.or_brute_knn_r.restype = ctypes.c_int
    L.or_brute_knn_rows.argtypes = [P, i64, i32, P, P, i64, i32, P, P, i32]
    L.or_brute_knn_rows.restype = ctypes.c_int
    L.or_max_depth.restype = i32
    L.or_sample_count.restype = i32
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int):
    if st != 0:
        raise OracleError(f"oracle: {STATUS.get(st, st)}")


def max_depth() -> int:
    return int(_load().or_max_depth())


def sample_count() -> int:
    return int(_load().or_sample_count())


class Tree:
    """Oracle kd-tree (owns a C handle)."""

    def __init__(self, handle, n: int, d: int, bucket: int, lib=None):
        self._h = handle
        self._L = lib if lib is not None else _lib
        self.n, self.d, self.bucket = n, d, bucket

    def __del__(self):
        h = getattr(self, "_h", None)
        L = getattr(self, "_L", None)
        if h and L is not None:
            L.or_free(h)
            self._h = None

    @property
    def num_nodes(self) -> int:
        return int(self._L.or_tree_num_nodes(self._h))

    @property
    def depth(self) -> int:
        return int(self._L.or_tree_depth(self._h))

    def export(self) -> dict:
        """Node table in preorder plus the leaf-order permutation."""
        nn, d = self.num_nodes, self.d
        meta = np.empty((nn, 4), np.int32)
        split = np.empty(nn, np.float32)
        rng = np.empty((nn, 4), np.int64)
        lo = np.empty((nn, d), np.float32)
        hi = np.empty((nn, d), np.float32)
        perm = np.empty(self.n, np.int32)
        self._L.or_tree_export(self._h, _ptr(meta), _ptr(split), _ptr(rng), _ptr(lo), _ptr(hi), _ptr(perm))
        return dict(leaf=meta[:, 0].astype(bool), index_split=meta[:, 1].astype(bool),
                    dim=meta[:, 2].copy(), depth=meta[:, 3].copy(), split=split,
                    start=rng[:, 0].copy(), count=rng[:, 1].copy(), left=rng[:, 2].copy(),
                    right=rng[:, 3].copy(), lo=lo, hi=hi, perm=perm)


def build(points: np.ndarray, bucket: int = 32, lib=None) -> Tree:
    """kd-tree over host points [n][d] (float32).  `lib`: a library from
    compile_variant (tests of planted mistakes); the oracle by default."""
    L = lib if lib is not None else _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    if pts.ndim != 2:
        raise ValueError("points must be [n][d]")
    n, d = pts.shape
    h = ctypes.c_void_p()
    _check(L.or_build(_ptr(pts), n, d, int(bucket), ctypes.byref(h)))
    return Tree(h, n, d, bucket, L)


def knn(tree: Tree, queries: np.ndarray, k: int, threads: int = 0, visits: bool = False, max_d2=None):
    """Algorithm 1 (corrected) for every query row; returns (ids, d2[, visits]).
    max_d2: Algorithm 1's radius r, squared (neighbours with d2 <= max_d2 only)."""
    q = np.ascontiguousarray(queries, dtype=np.float32)
    m = q.shape[0]
    if q.ndim != 2 or (m and q.shape[1] != tree.d):
        raise ValueError("queries must be [m][d]")
    ids = np.empty((m, k), np.int32)
    d2 = np.empty((m, k), np.float32)
    v = np.empty((m, 2), np.int64) if visits else None
    r2 = np.float32(np.inf if max_d2 is None else max_d2)
    _check(tree._L.or_knn_r(tree._h, _ptr(q), m, int(k), ctypes.c_float(r2), _ptr(ids), _ptr(d2),
                         _ptr(v) if v is not None else None, int(threads)))
    return (ids, d2, v) if visits else (ids, d2)


def brute_knn(points: np.ndarray, queries: np.ndarray, k: int, threads: int = 0, rows=None, max_d2=None):
    """Exhaustive KNN (the plain definition).  ``rows`` selects query rows;
    ``max_d2`` keeps only points with d2 <= max_d2."""
    L = _load()
    pts = np.ascontiguousarray(points, dtype=np.float32)
    q = np.ascontiguousarray(queries, dtype=np.float32)
    n, d = pts.shape
    if max_d2 is not None:
        if rows is not None:
            q = q[np.asarray(rows)]
        m = q.shape[0]
        ids = np.empty((m, k), np.int32)
        d2 = np.empty((m, k), np.float32)
        _check(L.or_brute_knn_r(_ptr(pts), n, d, _ptr(q), m, int(k), ctypes.c_float(np.float32(max_d2)),
                                _ptr(ids), _ptr(d2), int(threads)))
        return ids, d2
    if rows is None:
        m = q.shape[0]
        ids = np.empty((m, k), np.int32)
        d2 = np.empty((m, k), np.float32)
        _check(L.or_brute_knn(_ptr(pts), n, d, _ptr(q), m, int(k), _ptr(ids), _ptr(d2), int(threads)))
    else:
        r = np.ascontiguousarray(rows, dtype=np.int64)
        ids = np.empty((r.size, k), np.int32)
        d2 = np.empty((r.size, k), np.float32)
        _check(L.or_brute_knn_rows(_ptr(pts), n, d, _ptr(q), _ptr(r), r.size, int(k), _ptr(ids),
                                   _ptr(d2), int(threads)))
    return ids, d2

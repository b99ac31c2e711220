"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (stated by the result contract): neighbour ids bit-exact, FP32 squared
distances identical to 0 ULP (compared as bit patterns), and the kd-tree
identical node by node (split dimension, split value, ranges, boxes, leaf
order).  Full-size workloads are checked on sampled queries against the
oracle's exhaustive search plus tree invariants.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1607_08220_gb300 import workloads
from tests import treecheck

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08220_gb300 import build_ext, panda
    build_ext.build()
    panda.load()
    return panda


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def gpu_knn(P, tree, q, k, order="leaf", transpose_max=0, traversal="auto"):
    import torch
    ids, d2 = P.knn(tree, dev(q), k, order=order, transpose_max=transpose_max, traversal=traversal)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), d2.cpu().numpy()


def assert_same_knn(ids, d2, eids, ed2):
    assert ids.shape == eids.shape
    bad = np.flatnonzero((ids != eids).any(axis=1))
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:5]}: {ids[bad[0]]} vs {eids[bad[0]]}"
    assert np.array_equal(d2.view(np.uint32), ed2.view(np.uint32)), "d2 not bit-identical"


def full_parity(P, pts, q, k, B, orders=("leaf",), brute_rows=None, shapes=(0, -1, 32)):
    t = P.build(dev(pts), B)
    ot = oracle.build(pts, B)
    g = t.export()
    o = ot.export()
    treecheck.assert_same_tree(g, o)
    assert t.info()["depth"] == ot.depth
    eids, ed2 = oracle.knn(ot, q, k)
    for order in orders:
        ids, d2 = gpu_knn(P, t, q, k, order)
        assert_same_knn(ids, d2, eids, ed2)
    for shape in shapes:     # both leaf-scan shapes (lanes = queries, lanes = points)
        ids, d2 = gpu_knn(P, t, q, k, orders[0], transpose_max=shape, traversal="packet")
        assert_same_knn(ids, d2, eids, ed2)
    for order in orders:     # each lane walking its own query
        ids, d2 = gpu_knn(P, t, q, k, order, traversal="per_query")
        assert_same_knn(ids, d2, eids, ed2)
    if brute_rows is not None:
        bi, bd = oracle.brute_knn(pts, q, k, rows=brute_rows)
        assert_same_knn(eids[brute_rows], ed2[brute_rows], bi, bd)
    return t, g


# ------------------------------------------------------------------ small config


def test_uniform_small_full_parity(P):
    w = workloads.uniform_small()
    t, g = full_parity(P, w.points, w.queries, w.k, w.bucket, orders=("leaf", "morton", "none"),
                       brute_rows=np.arange(0, 10000, 7))
    treecheck.check_invariants_fast(g, w.points, w.bucket)


def _edge_cases():
    rng = np.random.default_rng(11)
    yield "n1", rng.random((1, 3), dtype=np.float32), rng.random((5, 3), dtype=np.float32), 4, 32
    yield "single_bucket", rng.random((20, 3), dtype=np.float32), rng.random((40, 3), dtype=np.float32), 7, 32
    yield "n_lt_k", rng.random((5, 2), dtype=np.float32), rng.random((33, 2), dtype=np.float32), 9, 4
    yield "k_eq_n", rng.random((64, 3), dtype=np.float32), rng.random((70, 3), dtype=np.float32), 64, 8
    lat = workloads.lattice_points(5000, 3, seed=5, side=6)
    yield "lattice_ties", lat, workloads.lattice_points(333, 3, seed=6, side=6), 33, 16
    yield "identical", np.full((2000, 3), 0.25, np.float32), rng.random((50, 3), dtype=np.float32), 5, 8
    dup = np.repeat(rng.random((6, 3), dtype=np.float32), 700, axis=0)
    yield "heavy_dups", dup, dup[::97], 17, 32
    x = rng.random((3000, 4), dtype=np.float32)
    x[:, 2] = 0.5
    yield "constant_dim", x, rng.random((100, 4), dtype=np.float32), 12, 4
    z = np.zeros((4096, 1), np.float32)
    z[1::2] = 0.7
    z[0::2] = 0.1
    yield "sample_all_min", z, np.array([[0.3], [0.9], [0.1]], np.float32), 3, 256
    for d in (1, 2, 5, 7, 8, 9, 12, 16):
        yield f"gauss_d{d}", rng.standard_normal((6000, d)).astype(np.float32), \
            rng.standard_normal((257, d)).astype(np.float32), 10, 32
    for k in (1, 8, 9, 16, 17, 32, 33, 64):
        yield f"k{k}", rng.random((9000, 3), dtype=np.float32), rng.random((100, 3), dtype=np.float32), k, 32
    for B in (1, 2, 5, 64, 256):
        yield f"B{B}", rng.random((5000, 3), dtype=np.float32), rng.random((99, 3), dtype=np.float32), 6, B
    # every strided sample of the root in the lowest (highest) quarter of the
    # split dimension's values: c_j crosses n/2 outside the window of interval
    # points the first histogram pass counts, and the root takes the full pass
    m = 40
    for name, base in (("window_miss_below", 0.0), ("window_miss_above", 0.75)):
        x = rng.random((1024 * m, 3), dtype=np.float32) * np.float32(0.1)
        u = rng.random(1024 * m, dtype=np.float32)
        on_sample = np.arange(1024 * m) % m == 0
        rest = np.float32(0.25) if base == 0.0 else np.float32(0.0)
        x[:, 0] = np.where(on_sample, np.float32(base) + np.float32(0.25) * u, rest + np.float32(0.75) * u)
        yield name, x, rng.random((300, 3), dtype=np.float32), 6, 32
    yield "neg_zero", np.array([[-0.0, 1.0], [0.0, 1.0], [0.0, -0.0], [-0.0, 0.0], [1.0, 1.0]] * 20,
                               np.float32), np.array([[0.0, 0.0], [-0.0, 0.5]], np.float32), 7, 4
    # hand-worked nodes whose split dimension depends on the exact FP32
    # summation order of the sample variance (tests/golden/variance_order.json)
    with open(os.path.join(os.path.dirname(__file__), "golden", "variance_order.json")) as f:
        for node in json.load(f)["nodes"]:
            pts = np.array(node["points"], np.float32)
            yield f"variance_{node['name']}", pts, pts[::3].copy(), 5, node["bucket"]


@pytest.mark.parametrize("case", list(_edge_cases()), ids=lambda c: c[0])
def test_edge_case_parity(P, case):
    name, pts, q, k, B = case
    full_parity(P, pts, q, k, B, orders=("leaf", "morton", "none"),
                brute_rows=np.arange(q.shape[0]))


def _self_cases():
    rng = np.random.default_rng(21)
    w = workloads.uniform_small()
    yield "uniform_small", w.points, 5, 32
    yield "n_lt_k", rng.random((5, 2), dtype=np.float32), 9, 4
    yield "identical", np.full((2000, 3), 0.25, np.float32), 5, 8
    dup = np.repeat(rng.random((6, 3), dtype=np.float32), 700, axis=0)
    yield "heavy_dups", dup, 17, 32
    yield "lattice_ties", workloads.lattice_points(5000, 3, seed=5, side=6), 33, 16
    yield "gauss_d10", rng.standard_normal((20000, 10)).astype(np.float32), 16, 32
    yield "gauss_d16_k64", rng.standard_normal((3000, 16)).astype(np.float32), 64, 8
    yield "cosmo", workloads.cosmology_points(300_000, seed=12, halos=50), 10, 32


@pytest.mark.parametrize("case", list(_self_cases()), ids=lambda c: c[0])
def test_self_query_parity(P, case):
    """The all-points query equals panda_knn with queries = the points (and the
    oracle), for both traversal shapes and the blocking and host variants."""
    import torch
    name, pts, k, B = case
    t = P.build(dev(pts), B)
    ri, rd = gpu_knn(P, t, pts, k)
    ot = oracle.build(pts, B)
    eids, ed2 = oracle.knn(ot, pts, k)
    assert_same_knn(ri, rd, eids, ed2)
    for trav in ("auto", "per_query"):
        si, sd = P.knn_self(t, k, traversal=trav)
        torch.cuda.synchronize()
        assert_same_knn(si.cpu().numpy(), sd.cpu().numpy(), eids, ed2)
    si, sd = P.knn_self_sync(t, k)
    assert_same_knn(si.cpu().numpy(), sd.cpu().numpy(), eids, ed2)
    hi, hd = P.knn_self_host(t, k)
    assert_same_knn(hi, hd, eids, ed2)


def _radius_cases():
    rng = np.random.default_rng(41)
    w = workloads.uniform_small()
    yield "uniform_small", w.points, w.queries, 8, 32, (0.0, 2e-5, 1e-4, 1e-3)
    lat = workloads.lattice_points(5000, 3, seed=5, side=6)
    yield "lattice_ties", lat, workloads.lattice_points(333, 3, seed=6, side=6), 20, 16, \
        (0.0, 2.0 ** -8, 2 * 2.0 ** -8, 2.0 ** -6)
    dup = np.repeat(rng.random((6, 3), dtype=np.float32), 700, axis=0)
    yield "heavy_dups", dup, dup[::97], 17, 32, (0.0, 0.01)
    yield "gauss_d10", rng.standard_normal((20000, 10)).astype(np.float32), \
        rng.standard_normal((500, 10)).astype(np.float32), 16, 32, (1.0, 4.0)


@pytest.mark.parametrize("case", list(_radius_cases()), ids=lambda c: c[0])
def test_radius_parity(P, case):
    """Algorithm 1's search radius: only points with d2 <= max_d2, padded with
    (-1, +inf); equal to the oracle for both traversal shapes, the all-points
    query and the host variant."""
    import torch
    name, pts, q, k, B, radii = case
    t = P.build(dev(pts), B)
    ot = oracle.build(pts, B)
    for r2 in radii:
        eids, ed2 = oracle.knn(ot, q, k, max_d2=r2)
        for trav in ("packet", "per_query"):
            ids, d2 = P.knn(t, dev(q), k, traversal=trav, max_d2=r2)
            torch.cuda.synchronize()
            assert_same_knn(ids.cpu().numpy(), d2.cpu().numpy(), eids, ed2)
        hi, hd = P.knn_host(t, q, k, max_d2=r2)
        assert_same_knn(hi, hd, eids, ed2)
        sids, sd2 = oracle.knn(ot, pts, k, max_d2=r2)
        si, sd = P.knn_self(t, k, max_d2=r2)
        torch.cuda.synchronize()
        assert_same_knn(si.cpu().numpy(), sd.cpu().numpy(), sids, sd2)


def test_radius_errors(P):
    import torch
    pts = np.random.default_rng(0).random((1000, 3), dtype=np.float32)
    t = P.build(dev(pts), 32)
    for bad in (-1.0, float("nan")):
        with pytest.raises(P.PandaError) as e:
            P.knn(t, dev(pts[:10]), 4, max_d2=bad)
        assert e.value.status == 1
    prm = P._params("leaf", 0, "auto", 0.01)
    ids = torch.empty((10, 4), dtype=torch.int32, device="cuda")
    d2 = torch.empty((10, 4), dtype=torch.float32, device="cuda")
    vis = torch.zeros((10, 2), dtype=torch.int32, device="cuda")
    q = dev(pts[:10])
    import ctypes
    st = P.load().panda_knn_visits(t.handle, ctypes.c_void_p(q.data_ptr()), 10, 4, ctypes.c_void_p(ids.data_ptr()),
                                   ctypes.c_void_p(d2.data_ptr()), ctypes.c_void_p(vis.data_ptr()), None,
                                   ctypes.byref(prm), None)
    assert st == 3                                     # work counters: unbounded queries only
    ok = P.knn(t, dev(pts[:10]), 4, max_d2=0.0)[0]     # the library stays usable
    torch.cuda.synchronize()
    assert ok[:, 0].cpu().tolist() == list(range(10))


def test_self_host_async_pipelined(P):
    """Enqueue-only host results and stream-ordered frees, two steps in flight on
    two streams, then with the builds on a third, high-priority stream: every
    step's host results equal the blocking call's."""
    import torch
    pts = workloads.cosmology_points(120_000, seed=44, halos=20)
    pn = torch.from_numpy(pts).pin_memory().numpy()
    t = P.build_host(pn, 32)
    want_i, want_d = P.knn_self_host(t, 8)
    t.free()
    sts = [torch.cuda.Stream(), torch.cuda.Stream()]
    keep = [(torch.empty((pts.shape[0], 8), dtype=torch.int32).pin_memory(),
             torch.empty((pts.shape[0], 8), dtype=torch.float32).pin_memory()) for _ in range(4)]
    outs = [(a.numpy(), b.numpy()) for a, b in keep]     # views of the pinned tensors kept alive above
    for i in range(4):
        s = sts[i % 2]
        tt = P.build_host(pn, 32, stream=s)
        P.knn_self_host(tt, 8, stream=s, out=outs[i], wait=False)
        tt.free(stream=s)
    torch.cuda.synchronize()
    for oi, od in outs:
        assert_same_knn(oi, od, want_i, want_d)
    # builds on a high-priority stream, each query and free on one of two
    # normal-priority streams after an event on the build stream
    lo, hi = torch.cuda.Stream.priority_range()
    bs = torch.cuda.Stream(priority=hi)
    qs = [torch.cuda.Stream(priority=lo), torch.cuda.Stream(priority=lo)]
    for o in outs:
        o[0].fill(0)
    for i in range(4):
        tt = P.build_host(pn, 32, stream=bs)
        ev = torch.cuda.Event()
        ev.record(bs)
        qs[i % 2].wait_event(ev)
        P.knn_self_host(tt, 8, stream=qs[i % 2], out=outs[i], wait=False)
        tt.free(stream=qs[i % 2])
    torch.cuda.synchronize()
    for oi, od in outs:
        assert_same_knn(oi, od, want_i, want_d)


def test_phase_timing_many_levels(P):
    """Phase timing across a build with many level passes (event bookkeeping)."""
    pts = np.random.default_rng(4).random((3_000_000, 3), dtype=np.float32)
    P.set_phase_timing(True)
    try:
        t = P.build(dev(pts), 8)
        names = [p[0] for p in P.phase_times()]
        assert "level.partition" in names and "subtree" in names
        ids, d2 = gpu_knn(P, t, pts[:1000], 4)
        assert "query.traverse" in [p[0] for p in P.phase_times()]
    finally:
        P.set_phase_timing(False)
    assert np.all(ids[:, 0] == np.arange(1000))


def test_empty_query_batch(P):
    import torch
    pts = np.random.default_rng(0).random((100, 3), dtype=np.float32)
    t = P.build(dev(pts), 8)
    ids, d2 = P.knn(t, torch.empty((0, 3), dtype=torch.float32, device="cuda"), 5)
    assert ids.shape == (0, 5)


# ------------------------------------------------------------------ several levels and tiles


def test_multilevel_cosmology_parity(P):
    pts = workloads.cosmology_points(400_000, seed=9, halos=60)
    q = workloads.cosmology_points(30_001, seed=10, halos=60)
    t, g = full_parity(P, pts, q, 10, 32, orders=("leaf", "morton"), brute_rows=np.arange(0, 30001, 97))
    treecheck.check_invariants_fast(g, pts, 32)
    assert t.info()["depth"] <= treecheck.balance_bound(pts.shape[0], 32)


def test_lattice_duplicates_many_tiles(P):
    """2^21 points on a 24^3 lattice (about 150 copies of every position) plus
    a 2^20-point block of one repeated value: level passes over many tiles
    with heavy ties, splits where the value rule leaves nothing on one side
    (the duplicate fallback), nodes of identical points (index splits) and
    windows of equal interval points.  Tree identical to the oracle's node by
    node; sampled rows of a query set and of the all-points query against
    exhaustive search."""
    lat = workloads.lattice_points(1 << 21, 3, seed=41, side=24)
    same = np.full((1 << 20, 3), 0.5, np.float32)
    pts = np.concatenate([lat, same])[np.random.default_rng(42).permutation((1 << 21) + (1 << 20))]
    q = workloads.lattice_points(20_000, 3, seed=43, side=24)
    t = P.build(dev(pts), 32)
    ot = oracle.build(pts, 32)
    treecheck.assert_same_tree(t.export(), ot.export())
    rows = np.arange(0, q.shape[0], 41)
    ids, d2 = gpu_knn(P, t, q[rows], 12)
    bi, bd = oracle.brute_knn(pts, q[rows], 12)
    assert_same_knn(ids, d2, bi, bd)
    # the all-points query (walks down to each job's leaf by the inner headers)
    import torch
    si, sd = P.knn_self(t, 12)
    torch.cuda.synchronize()
    prow = np.arange(0, pts.shape[0], 4099)
    bi, bd = oracle.brute_knn(pts, pts, 12, rows=prow)
    assert_same_knn(si.cpu().numpy()[prow], sd.cpu().numpy()[prow], bi, bd)
    t.free()


def test_plasma_slab_parity(P):
    pts = workloads.plasma_points(300_000, seed=4)
    q = workloads.plasma_points(20_000, seed=7)
    full_parity(P, pts, q, 8, 32, orders=("leaf",), brute_rows=np.arange(0, 20000, 101))


def test_ten_dim_parity(P):
    w = workloads.features_10d(n=150_000, m=5_000)
    full_parity(P, w.points, w.queries, 16, 32, orders=("leaf", "morton"), brute_rows=np.arange(0, 5000, 23))


# ------------------------------------------------------------------ full sizes (launch config of the benchmark)


def test_cosmology_self_full_size(P):
    """n = 2^24 self-KNN, k = 10, B = 32: tree identical to the oracle's; 2,000
    sampled rows against exhaustive search; every point is its own rank-0
    neighbour unless an exact duplicate with a smaller id exists."""
    import torch
    w = workloads.cosmology_self()
    t = P.build(dev(w.points), w.bucket)
    ids, d2 = P.knn(t, dev(w.points), w.k)
    torch.cuda.synchronize()
    ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
    g = t.export()
    treecheck.check_invariants_fast(g, w.points, w.bucket)
    assert t.info()["depth"] <= treecheck.balance_bound(w.points.shape[0], w.bucket)
    rows = np.random.default_rng(1).choice(w.points.shape[0], 2000, replace=False)
    bi, bd = oracle.brute_knn(w.points, w.points, w.k, rows=rows)
    assert_same_knn(ids[rows], d2[rows], bi, bd)
    assert np.all(d2[:, 0] == 0.0)
    u, first = np.unique(w.points, axis=0, return_index=True)
    nodup = np.ones(w.points.shape[0], bool)
    if u.shape[0] < w.points.shape[0]:
        nodup[:] = False
        nodup[first] = True
    assert np.all(ids[nodup, 0] == np.flatnonzero(nodup))
    ot = oracle.build(w.points, w.bucket)
    treecheck.assert_same_tree(g, ot.export())
    si, sd = P.knn_self(t, w.k)              # the all-points query: the same rows
    torch.cuda.synchronize()
    assert_same_knn(si.cpu().numpy(), sd.cpu().numpy(), ids, d2)


def test_sparse_queries_full_size_tree(P):
    """Few queries against the 2^24-point tree (the automatic choice walks each
    query on its own lane): equal to the packet traversal and, on sampled rows,
    to exhaustive search."""
    import torch
    w = workloads.cosmology_self()
    q = workloads.cosmology_points(60_000, seed=77)
    t = P.build(dev(w.points), w.bucket)
    res = {}
    for trav in ("auto", "per_query", "packet"):
        ids, d2 = P.knn(t, dev(q), 16, traversal=trav)
        torch.cuda.synchronize()
        res[trav] = (ids.cpu().numpy(), d2.cpu().numpy())
    assert_same_knn(*res["auto"], *res["packet"])
    assert_same_knn(*res["per_query"], *res["packet"])
    rows = np.random.default_rng(3).choice(q.shape[0], 300, replace=False)
    bi, bd = oracle.brute_knn(w.points, q, 16, rows=rows)
    assert_same_knn(res["auto"][0][rows], res["auto"][1][rows], bi, bd)


def test_features_10d_full_size(P):
    import torch
    w = workloads.features_10d()
    t = P.build(dev(w.points), 32)
    ids, d2 = P.knn(t, dev(w.queries), w.k)
    torch.cuda.synchronize()
    ids, d2 = ids.cpu().numpy(), d2.cpu().numpy()
    rows = np.random.default_rng(2).choice(w.queries.shape[0], 600, replace=False)
    bi, bd = oracle.brute_knn(w.points, w.queries, w.k, rows=rows)
    assert_same_knn(ids[rows], d2[rows], bi, bd)
    treecheck.check_invariants_fast(t.export(), w.points, 32)


# ------------------------------------------------------------------ API surface


def test_host_variants_match(P):
    w = workloads.uniform_small(n=50_000, m=3_000)
    t = P.build_host(w.points, 32)
    ids, d2 = P.knn_host(t, w.queries, 5)
    t2 = P.build(dev(w.points), 32)
    gi, gd = gpu_knn(P, t2, w.queries, 5)
    assert_same_knn(ids, d2, gi, gd)
    si, sd = P.knn_sync(t2, dev(w.queries), 5)
    assert_same_knn(si.cpu().numpy(), sd.cpu().numpy(), gi, gd)


def test_concurrent_streams_same_tree(P):
    import torch
    w = workloads.uniform_small(n=200_000, m=40_000)
    t = P.build(dev(w.points), 32)
    q = dev(w.queries)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        a = P.knn(t, q, 9, stream=s1)
    with torch.cuda.stream(s2):
        b = P.knn(t, q, 9, stream=s2, order="morton")
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))


def test_errors_are_reported(P):
    import torch
    bad = np.random.default_rng(0).random((1000, 3), dtype=np.float32)
    bad[17, 1] = np.nan
    with pytest.raises(P.PandaError) as e:
        P.build(dev(bad), 32)
    assert e.value.status == 2
    good = np.random.default_rng(1).random((1000, 3), dtype=np.float32)
    t = P.build(dev(good), 32)
    q = good[:50].copy()
    q[3, 0] = np.inf
    with pytest.raises(P.PandaError) as e:
        P.knn_sync(t, dev(q), 4)
    assert e.value.status == 2
    with pytest.raises(P.PandaError) as e:
        P.knn(t, dev(good[:10]), 65)
    assert e.value.status == 3
    import ctypes
    L = P.load()
    h = ctypes.c_void_p()
    host = np.ascontiguousarray(good)
    st = L.panda_build(host.ctypes.data_as(ctypes.c_void_p), 1000, 3, 32, ctypes.byref(h))
    assert st == 1     # host pointer given to the device entry point
    # the library stays usable after each error
    ids, d2 = gpu_knn(P, t, good[:10], 3)
    assert np.all(ids[:, 0] == np.arange(10))

"""panda_knn_noalloc: the KNN entry point that allocates no device memory.

It exists for callers that cannot allocate while they query -- code running
under an allocator it does not own, or on a path that must never wait on or
fail in an allocation.  Its scratch space is a fixed array inside the library,
so this test checks, through the C ABI, that two calls in a row return exactly
what panda_knn_async returns (same ids, same distance bits: the tolerance of
every parity test here), and that sizes beyond the fixed limit are refused.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_knn_async_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_1607_08220_gb300 import build_ext, panda as P, workloads
    build_ext.build()
    L = P.load()
    pts = workloads.cosmology_points(300_000, seed=21, halos=40)
    tree = P.build(torch.from_numpy(pts).cuda(), 32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for m, k, seed in [(70_001, 10, 22), (50_000, 7, 23)]:
        q = torch.from_numpy(workloads.cosmology_points(m, seed=seed, halos=40)).cuda()
        ref_ids, ref_d2 = P.knn(tree, q, k)
        ids = torch.full((m, k), -7, dtype=torch.int32, device="cuda")
        d2 = torch.full((m, k), -7.0, dtype=torch.float32, device="cuda")
        st = L.panda_knn_noalloc(tree.handle, ctypes.c_void_p(q.data_ptr()), m, k,
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()), stream)
        assert st == 0, L.panda_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        assert torch.equal(d2.view(torch.int32), ref_d2.view(torch.int32))
    # the branch without an ordering pass (m <= 32), the limit itself (m = 2^20:
    # the whole scratch array, a bin shift other than panda_knn_async's), a
    # small tree with more queries than half its points, and a 10-D tree (the
    # wide-point traversal): each through the C ABI against panda_knn_async
    rng = np.random.default_rng(24)
    small = P.build(torch.from_numpy(workloads.cosmology_points(5_000, seed=25, halos=4)).cuda(), 32)
    feat = workloads.features_10d(n=60_000, m=4_000)
    wide = P.build(torch.from_numpy(feat.points).cuda(), 32)
    cases = [(tree, torch.from_numpy(workloads.cosmology_points(17, seed=26, halos=40)).cuda(), 5),
             (tree, torch.from_numpy(workloads.cosmology_points(1 << 20, seed=27, halos=40)).cuda(), 8),
             (small, torch.from_numpy(workloads.cosmology_points(4_000, seed=28, halos=4)).cuda(), 12),
             (wide, torch.from_numpy(feat.queries).cuda(), 16),
             (tree, torch.from_numpy(rng.random((33, 3), dtype=np.float32)).cuda(), 1)]
    for t, q, k in cases:
        m = q.shape[0]
        ref_ids, ref_d2 = P.knn(t, q, k)
        ids = torch.full((m, k), -7, dtype=torch.int32, device="cuda")
        d2 = torch.full((m, k), -7.0, dtype=torch.float32, device="cuda")
        st = L.panda_knn_noalloc(t.handle, ctypes.c_void_p(q.data_ptr()), m, k,
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(d2.data_ptr()), stream)
        assert st == 0, L.panda_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids), (m, k)
        assert torch.equal(d2.view(torch.int32), ref_d2.view(torch.int32)), (m, k)
    # more queries than the fixed scratch holds: refused with a clear error
    q = torch.zeros((8, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((8, 4), dtype=torch.int32, device="cuda")
    st = L.panda_knn_noalloc(tree.handle, ctypes.c_void_p(q.data_ptr()), (1 << 20) + 1, 4,
                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 3 and b"limit" in L.panda_last_error()

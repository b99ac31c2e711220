"""Host-side fault injection: a device allocation that fails inside a call.

Every synchronous entry point is run with an injected allocation failure at
each of its workspace allocations in turn (panda_debug_fail_alloc).  Each
such call must return PANDA_ERR_OUT_OF_MEMORY, hold no device memory
afterwards (the stream-ordered pool's bytes in use are what they were before
the call) and leave the library usable; once the injection point lies past
the call's last allocation the call succeeds with the same result as without
injection.  No GPU fault is involved: the failure is made on the host.  The
file runs after the other GPU tests (its name), so that a failure here stops
none of them under -x (only the allocation-free entry point's test comes later).

The byte count is the library's own count of its live allocations
(panda_debug_pool_used), and the garbage collector is off during a sweep:
a tree that an earlier test left to the collector would otherwise be freed
in the middle of a sweep and lower the count by memory the swept call never
held."""
import gc

import numpy as np
import pytest

from paper_1607_08220_gb300 import workloads

pytestmark = pytest.mark.gpu

OOM = 4


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08220_gb300 import build_ext, panda
    build_ext.build()
    panda.load()
    yield panda
    panda.debug_fail_alloc(-1)


def sweep(P, call, max_allocs=128):
    """Fail allocation 0, 1, 2, ... of `call` until it succeeds; returns its
    result and how many allocations it made."""
    import torch
    gc.collect()
    torch.cuda.synchronize()
    was_enabled = gc.isenabled()
    gc.disable()
    base = P.debug_pool_used()
    try:
        for j in range(max_allocs):
            P.debug_fail_alloc(j)
            try:
                out = call()
            except P.PandaError as e:
                assert e.status == OOM, (j, e.status, str(e))
                assert "injected" in str(e), str(e)
                assert P.debug_pool_used() == base, f"allocation {j} failed: device memory left held"
                continue
            torch.cuda.synchronize()
            return out, j
        raise AssertionError(f"still failing after {max_allocs} injected failures")
    finally:
        P.debug_fail_alloc(-1)
        if was_enabled:
            gc.enable()


def same(a, b):
    import torch
    torch.cuda.synchronize()
    return torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))


def test_build_and_queries_fail_cleanly(P):
    import torch
    pts = workloads.cosmology_points(200_000, seed=61, halos=30)
    pd = torch.from_numpy(pts).cuda()
    t, nalloc = sweep(P, lambda: P.build(pd, 32))
    assert nalloc >= 20           # level-stage scratch, then the tree tables
    ref = P.build(pd, 32)
    want = P.knn_self(ref, 8)
    assert same(P.knn_self(t, 8), want)

    got, nalloc = sweep(P, lambda: P.knn_self(t, 8))
    assert nalloc >= 1 and same(got, want)

    q = torch.from_numpy(workloads.cosmology_points(20_000, seed=62, halos=30)).cuda()
    want_q = P.knn(ref, q, 7)
    for order in ("leaf", "morton", "none"):
        got, nalloc = sweep(P, lambda: P.knn(t, q, 7, order=order))
        assert nalloc >= 1 and same(got, want_q), order

    t.free()
    ref.free()


def test_host_variants_fail_cleanly(P):
    import torch
    pts = workloads.cosmology_points(100_000, seed=63, halos=20)
    qs = workloads.cosmology_points(5_000, seed=64, halos=20)
    t, nalloc = sweep(P, lambda: P.build_host(pts, 32))
    assert nalloc >= 21           # the staging copy of the points comes first
    ref = P.build(torch.from_numpy(pts).cuda(), 32)
    (gi, gd), _ = sweep(P, lambda: P.knn_host(t, qs, 5))
    wi, wd = P.knn(ref, torch.from_numpy(qs).cuda(), 5)
    torch.cuda.synchronize()
    assert np.array_equal(gi, wi.cpu().numpy()) and np.array_equal(gd.view(np.uint32), wd.cpu().numpy().view(np.uint32))
    (si, sd), _ = sweep(P, lambda: P.knn_self_host(t, 6))
    ri, rd = P.knn_self(ref, 6)
    torch.cuda.synchronize()
    assert np.array_equal(si, ri.cpu().numpy()) and np.array_equal(sd.view(np.uint32), rd.cpu().numpy().view(np.uint32))
    t.free()
    ref.free()


def test_refit_fails_cleanly_and_keeps_the_tree(P):
    import torch
    p0 = workloads.cosmology_points(50_000, seed=65, halos=10)
    t = P.build(torch.from_numpy(p0).cuda(), 32)
    before = P.knn_self(t, 4)
    rng = np.random.default_rng(66)
    p1 = (p0 + rng.standard_normal(p0.shape).astype(np.float32) * np.float32(0.002)).astype(np.float32)
    p1d = torch.from_numpy(p1).cuda()
    P.debug_fail_alloc(0)
    with pytest.raises(P.PandaError) as e:
        P.refit(t, p1d)
    P.debug_fail_alloc(-1)
    assert e.value.status == OOM
    assert same(P.knn_self(t, 4), before)      # nothing moved
    _, nalloc = sweep(P, lambda: P.refit(t, p1d))
    assert nalloc == 1
    fresh = P.build(p1d, 32)
    assert same(P.knn_self(t, 4), P.knn_self(fresh, 4))

"""Autotuner: picks a valid (bucket, order, traversal, scan shape) by timing, caches it, and
the tuned configuration returns exactly the CPU oracle's answer (and the default
configuration's: none of the knobs may change an answer)."""
import numpy as np
import pytest

import oracle
from paper_1607_08220_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_tune_choice_is_exact_and_cached():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_1607_08220_gb300 import build_ext, panda as P
    build_ext.build()
    P.load()
    np_pts = workloads.cosmology_points(200_000, seed=70, halos=30)
    np_q = workloads.cosmology_points(30_000, seed=71, halos=30)
    pts, q = torch.from_numpy(np_pts).cuda(), torch.from_numpy(np_q).cuda()
    r = P.tune(pts, q[:20_000], k=10, m_total=200_000)
    assert r["bucket"] in (16, 32, 64) and r["order"] in ("none", "morton", "leaf")
    assert r["traversal"] in ("packet", "per_query")
    assert r["transpose_max"] in ((-1, 4, 8, 12, 16, 32) if r["traversal"] == "packet" else (0,))
    assert r["score_ms"] > 0 and r["score_ms"] >= r["build_ms"]
    assert P.tune_lookup(3, 200_000, 10, 200_000) == r
    assert P.tune_lookup(3, 200_000, 11, 200_000) is None
    tuned = P.build(pts, r["bucket"])
    ti, td = P.knn(tuned, q, 10, order=r["order"], transpose_max=r["transpose_max"], traversal=r["traversal"])
    default = P.build(pts, 32)
    di, dd = P.knn(default, q, 10)
    torch.cuda.synchronize()
    ei, ed = oracle.knn(oracle.build(np_pts, r["bucket"]), np_q, 10)
    assert np.array_equal(ti.cpu().numpy(), ei)
    assert np.array_equal(td.cpu().numpy().view(np.uint32), ed.view(np.uint32))
    assert torch.equal(ti, di) and torch.equal(td.view(torch.int32), dd.view(torch.int32))
    # every other candidate the tuner times is exact too: each bucket size x
    # traversal shape against the oracle on a sample of the queries
    sub = np_q[:3000]
    ei, ed = oracle.knn(oracle.build(np_pts, 32), sub, 10)
    for B in (16, 32, 64):
        tb = P.build(pts, B)
        for kw in (dict(order="morton", traversal="packet", transpose_max=4),
                   dict(order="leaf", traversal="packet", transpose_max=32),
                   dict(order="none", traversal="per_query")):
            gi, gd = P.knn(tb, torch.from_numpy(sub).cuda(), 10, **kw)
            torch.cuda.synchronize()
            assert np.array_equal(gi.cpu().numpy(), ei), (B, kw)
            assert np.array_equal(gd.cpu().numpy().view(np.uint32), ed.view(np.uint32)), (B, kw)

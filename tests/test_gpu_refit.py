"""Refit (moved particles, same tree structure): every box is tight for the
new coordinates and queries on the refitted tree return exactly the KNN of
the new points (the answer is unique, so it equals a fresh build's and
exhaustive search's)."""
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


def moved(pts, seed, scale):
    rng = np.random.default_rng(seed)
    return (pts + rng.standard_normal(pts.shape).astype(np.float32) * np.float32(scale)).astype(np.float32)


@pytest.mark.parametrize("d", [3, 10])
def test_refit_exact_after_motion(P, d):
    import torch
    if d == 3:
        p0 = workloads.cosmology_points(200_000, seed=90, halos=40)
        steps = (0.001, 0.01)
    else:
        p0 = workloads.features_10d(n=60_000, m=1).points
        steps = (0.05, 0.3)
    t = P.build(torch.from_numpy(p0).cuda(), 32)
    p = p0
    for i, sc in enumerate(steps):
        p = moved(p, 100 + i, sc)
        pd = torch.from_numpy(p).cuda()
        P.refit(t, pd)
        treecheck.check_boxes(t.export(), p)
        si, sd = P.knn_self(t, 10)
        fresh = P.build(pd, 32)
        fi, fd = P.knn_self(fresh, 10)
        torch.cuda.synchronize()
        assert torch.equal(si, fi) and torch.equal(sd.view(torch.int32), fd.view(torch.int32))
        rows = np.random.default_rng(i).choice(p.shape[0], 300, replace=False)
        bi, bd = oracle.brute_knn(p, p, 10, rows=rows)
        assert np.array_equal(si.cpu().numpy()[rows], bi)
        assert np.array_equal(sd.cpu().numpy()[rows].view(np.uint32), bd.view(np.uint32))
        q = moved(p[:2000], 200 + i, 0.01 if d == 3 else 0.2)      # general queries too
        gi, gd = P.knn(t, torch.from_numpy(q).cuda(), 7)
        ri, rd = P.knn(fresh, torch.from_numpy(q).cuda(), 7)
        torch.cuda.synchronize()
        assert torch.equal(gi, ri) and torch.equal(gd.view(torch.int32), rd.view(torch.int32))


def test_refit_rejects_nonfinite_and_keeps_tree(P):
    import torch
    p0 = np.random.default_rng(5).random((5000, 3), dtype=np.float32)
    t = P.build(torch.from_numpy(p0).cuda(), 16)
    before = P.knn_self(t, 4)
    bad = p0.copy()
    bad[77, 2] = np.inf
    with pytest.raises(P.PandaError) as e:
        P.refit(t, torch.from_numpy(bad).cuda())
    assert e.value.status == 2
    after = P.knn_self(t, 4)
    torch.cuda.synchronize()
    assert torch.equal(before[0], after[0]) and torch.equal(before[1], after[1])
    treecheck.check_boxes(t.export(), p0)

"""KNN prediction (Sec. I: majority vote / average of the neighbours' values)
on the GPU equals the CPU oracle bit for bit, on KNN results of the general
and the all-points query, with padding (n < k) and k up to 64."""
import numpy as np
import pytest

import oracle
from oracle import predict
from paper_1607_08220_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1607_08220_gb300 import build_ext, panda
    build_ext.build()
    panda.load()
    return panda


def rule_labels(x):
    return ((x[:, 0] > 0).astype(np.int32) + 2 * (x[:, 1] > 0.2).astype(np.int32)).astype(np.int32)


@pytest.mark.parametrize("k", [1, 7, 16, 64])
def test_vote_and_mean_match_oracle(P, k):
    import torch
    w = workloads.features_10d(n=60_000, m=5_000)
    pts, q = w.points, w.queries
    labels = rule_labels(pts)
    values = (pts[:, 2] + np.float32(3.0) * pts[:, 3]).astype(np.float32)
    t = P.build(torch.from_numpy(pts).cuda(), 32)
    ids, _ = P.knn(t, torch.from_numpy(q).cuda(), k)
    lab_d, val_d = torch.from_numpy(labels).cuda(), torch.from_numpy(values).cuda()
    gv = P.knn_vote(ids, lab_d)
    gm = P.knn_mean(ids, val_d)
    torch.cuda.synchronize()
    h = ids.cpu().numpy()
    assert np.array_equal(gv.cpu().numpy(), predict.knn_vote(h, labels))
    assert np.array_equal(gm.cpu().numpy().view(np.uint32), predict.knn_mean(h, values).view(np.uint32))
    # the neighbours the oracle's tree finds give the same predictions
    ot = oracle.build(pts, 32)
    eids, _ = oracle.knn(ot, q, k)
    assert np.array_equal(predict.knn_vote(eids, labels), gv.cpu().numpy())
    if k >= 7:
        # the rule is learnable: nearest-neighbour votes recover most query labels
        assert (gv.cpu().numpy() == rule_labels(q)).mean() > 0.8


def test_padding_and_self_query(P):
    import torch
    rng = np.random.default_rng(9)
    pts = rng.random((5, 3), dtype=np.float32)
    labels = np.array([4, 4, 1, 1, 9], np.int32)
    values = np.array([1.0, 2.0, 3.0, 4.0, 5.0], np.float32)
    t = P.build(torch.from_numpy(pts).cuda(), 4)
    ids, _ = P.knn_self(t, 9)             # 9 > n = 5: four -1 entries per row
    gv = P.knn_vote(ids, torch.from_numpy(labels).cuda())
    gm = P.knn_mean(ids, torch.from_numpy(values).cuda())
    torch.cuda.synchronize()
    h = ids.cpu().numpy()
    assert (h[:, 5:] == -1).all()
    assert gv.cpu().numpy().tolist() == [1] * 5          # counts 4:2, 1:2, 9:1 -> tie -> 1
    assert np.array_equal(gm.cpu().numpy().view(np.uint32), predict.knn_mean(h, values).view(np.uint32))
    empty = torch.full((3, 4), -1, dtype=torch.int32, device="cuda")
    assert P.knn_vote(empty, torch.from_numpy(labels).cuda()).cpu().tolist() == [-1, -1, -1]
    assert torch.isnan(P.knn_mean(empty, torch.from_numpy(values).cuda())).all()

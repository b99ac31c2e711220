"""Pins of the KNN prediction oracle (Sec. I: majority vote / average of the
neighbours' values) against hand-worked rows and independent library routines."""
import numpy as np
import pytest

from oracle import predict


def test_vote_hand_worked_rows():
    labels = np.array([0, 1, 1, 2, 2, 7], np.int32)
    ids = np.array([[3, 1, 4, -1],     # labels 2, 1, 2 -> 2
                    [1, 3, -1, -1],    # labels 1, 2 tie -> smallest, 1
                    [-1, -1, -1, -1],  # no neighbour -> -1
                    [5, 0, 5, 0],      # 7, 0, 7, 0 tie -> 0
                    [5, 5, 5, 2]], np.int32)
    assert predict.knn_vote(ids, labels).tolist() == [2, 1, -1, 0, 7]


def test_mean_hand_worked_rows():
    values = np.array([0.5, 1.0, 2.0, -4.0], np.float32)
    ids = np.array([[0, 1, 2], [3, -1, -1], [-1, -1, -1], [0, 0, 3]], np.int32)
    out = predict.knn_mean(ids, values)
    assert out[0] == np.float32(3.5 / 3)
    assert out[1] == np.float32(-4.0)
    assert np.isnan(out[2])
    assert out[3] == np.float32(-1.0)


def test_mean_rank_order_rounding():
    # 2^24 + 1 + 1 in FP32 rank order: each +1 is lost to rounding, unlike the exact mean
    values = np.array([2.0 ** 24, 1.0, 1.0], np.float32)
    out = predict.knn_mean(np.array([[0, 1, 2]], np.int32), values)
    assert out[0] == np.float32(np.float32(2.0 ** 24) / np.float32(3.0))
    out2 = predict.knn_mean(np.array([[1, 2, 0]], np.int32), values)   # 1 + 1 first: exact
    assert out2[0] == np.float32(np.float32(2.0 ** 24 + 2) / np.float32(3.0))


def test_vote_matches_scipy_mode():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    labels = rng.integers(0, 5, 2000).astype(np.int32)
    ids = rng.integers(0, 2000, (500, 9)).astype(np.int32)
    want = stats.mode(labels[ids], axis=1, keepdims=False).mode   # smallest of the modes
    assert np.array_equal(predict.knn_vote(ids, labels), want.astype(np.int32))


def test_mean_close_to_fp64_mean():
    rng = np.random.default_rng(4)
    values = rng.standard_normal(5000).astype(np.float32)
    ids = rng.integers(-1, 5000, (400, 16)).astype(np.int32)
    out = predict.knn_mean(ids, values).astype(np.float64)
    for r in range(ids.shape[0]):
        v = ids[r][ids[r] >= 0]
        if v.size == 0:
            assert np.isnan(out[r])
            continue
        exact = values[v].astype(np.float64).mean()
        bound = (v.size + 1) * 2.0 ** -24 * np.abs(values[v]).astype(np.float64).sum() / v.size + 1e-30
        assert abs(out[r] - exact) <= bound

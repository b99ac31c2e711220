"""Test-side kd-tree checks written independently of both implementations (numpy only).

A tree is handled in a canonical preorder form (dict of numpy arrays): leaf,
index_split, dim, split, start, count, left, right (child positions in the same
preorder arrays, -1 for leaves), lo, hi ([nodes][d] tight boxes), perm (leaf
order of the original row ids) and depth.

Invariants (from Sec. III-A of the paper and the split rule the build follows):
  * the leaf order is a permutation of the input rows;
  * every leaf holds at most B points, every inner node more than B;
  * children partition their parent's range, left then right;
  * every point lies on the correct side of every ancestor split
    (x[dim] < s on the left, x[dim] >= s on the right), except below an index
    split, whose points are all identical;
  * every box is the exact min/max of the node's points.
"""
from __future__ import annotations

import math

import numpy as np


def canonical_from_oracle(exp: dict) -> dict:
    return dict(exp)


def check_invariants(t: dict, points: np.ndarray, bucket: int):
    pts = np.asarray(points, np.float32)
    n, d = pts.shape
    perm = np.asarray(t["perm"])
    assert perm.shape == (n,)
    assert np.array_equal(np.sort(perm), np.arange(n)), "leaf order is not a permutation"
    P = pts[perm]                     # points in leaf order
    nn = len(t["leaf"])
    assert t["start"][0] == 0 and t["count"][0] == n
    for i in range(nn):
        s, c = int(t["start"][i]), int(t["count"][i])
        assert c >= 1
        seg = P[s:s + c]
        assert np.array_equal(t["lo"][i], seg.min(axis=0)), f"box lo of node {i} not tight"
        assert np.array_equal(t["hi"][i], seg.max(axis=0)), f"box hi of node {i} not tight"
        if t["leaf"][i]:
            assert c <= bucket, f"leaf {i} holds {c} > B={bucket}"
            continue
        assert c > bucket, f"inner node {i} holds {c} <= B"
        l, r = int(t["left"][i]), int(t["right"][i])
        assert t["start"][l] == s and t["start"][r] == s + t["count"][l]
        assert t["count"][l] + t["count"][r] == c and t["count"][l] >= 1 and t["count"][r] >= 1
        assert t["depth"][l] == t["depth"][i] + 1 and t["depth"][r] == t["depth"][i] + 1
        if t["index_split"][i]:
            assert np.all(seg == seg[0]), f"index split {i} over non-identical points"
            assert t["count"][l] == (c + 1) // 2
        else:
            k, sv = int(t["dim"][i]), np.float32(t["split"][i])
            cl = int(t["count"][l])
            assert np.all(seg[:cl, k] < sv), f"node {i}: left point >= split"
            assert np.all(seg[cl:, k] >= sv), f"node {i}: right point < split"
    # stability: a node's points keep input order, so ids inside a leaf increase
    for i in np.flatnonzero(t["leaf"]):
        s, c = int(t["start"][i]), int(t["count"][i])
        assert np.all(np.diff(perm[s:s + c]) > 0), f"leaf {i} not in stable order"


def balance_bound(n: int, bucket: int) -> int:
    """Depth allowed for a near-balanced tree: ceil(log2(n/B)) + 2 (cf. depth 21 for 50M at B=32)."""
    if n <= bucket:
        return 0
    return int(math.ceil(math.log2(n / bucket))) + 2


def sample_positions(count: int, S: int = 1024) -> np.ndarray:
    s = min(S, count)
    return (np.arange(s, dtype=np.int64) * count) // s


def check_split_dim(t: dict, points: np.ndarray, node: int, S: int = 1024, rtol: float = 1e-4):
    """Max-variance dimension over the sample (Sec. III-A1), variance taken in fp64.

    Returns False (not checked) when the top two variances are within rtol, where
    FP32 rounding may legitimately pick either, or when the sample is constant
    along the fp64 winner (the duplicate fallback then applies)."""
    pts = np.asarray(points, np.float32)
    s, c = int(t["start"][node]), int(t["count"][node])
    rows = np.sort(t["perm"][s:s + c])[sample_positions(c, S)]
    var = pts[rows].astype(np.float64).var(axis=0)
    order = np.argsort(-var, kind="stable")
    if var[order[0]] == 0.0 or np.unique(pts[rows, order[0]]).size < 2:
        return False
    if len(var) > 1 and var[order[1]] >= var[order[0]] * (1 - rtol):
        return False
    assert int(t["dim"][node]) == int(order[0]), (node, t["dim"][node], var)
    return True


def check_split_rule(t: dict, points: np.ndarray, node: int, S: int = 1024):
    """The split of one value-split node is the sample value whose count of
    strictly smaller node points is closest to half the node (ties -> smaller value),
    counted here with searchsorted over the sorted node column."""
    pts = np.asarray(points, np.float32)
    P = pts[t["perm"]]
    s, c = int(t["start"][node]), int(t["count"][node])
    k = int(t["dim"][node])
    col = np.sort(P[s:s + c, k])
    vals = _presplit_column(t, pts, node)[sample_positions(c, S)]
    below = np.searchsorted(col, vals, side="left")        # #{x < v}
    err = np.abs(2 * below - c)
    best = err.min()
    cand = vals[err == best]
    expect = cand.min()
    assert np.float32(t["split"][node]) == expect, (node, t["split"][node], expect)


def _presplit_column(t: dict, pts: np.ndarray, node: int) -> np.ndarray:
    """Column of the node's own split dim in the node's stable (pre-split) order.

    Every partition is stable, so the order of a node's points is the order of
    the root's input restricted to the node: sort the node's original row ids.
    """
    s, c = int(t["start"][node]), int(t["count"][node])
    rows = np.sort(t["perm"][s:s + c])
    return pts[rows, int(t["dim"][node])]



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




def check_invariants_fast(t: dict, points: np.ndarray, bucket: int):
    """Vectorised form of check_invariants for large trees (one numpy pass per depth)."""
    pts = np.asarray(points, np.float32)
    n, d = pts.shape
    perm = np.asarray(t["perm"], np.int64)
    assert perm.shape == (n,) and perm.min() >= 0 and perm.max() < n
    assert np.all(np.bincount(perm, minlength=n) == 1), "leaf order is not a permutation"
    P = pts[perm]
    leaf = np.asarray(t["leaf"], bool)
    start, count = np.asarray(t["start"]), np.asarray(t["count"])
    left, right = np.asarray(t["left"]), np.asarray(t["right"])
    assert start[0] == 0 and count[0] == n
    assert np.all(count[leaf] <= bucket) and np.all(count[leaf] >= 1)
    inner = np.flatnonzero(~leaf)
    assert np.all(count[inner] > bucket)
    l, r = left[inner], right[inner]
    assert np.all(start[l] == start[inner]) and np.all(start[r] == start[inner] + count[l])
    assert np.all(count[l] + count[r] == count[inner]) and np.all(count[l] >= 1) and np.all(count[r] >= 1)
    dep = np.asarray(t["depth"])
    assert np.all(dep[l] == dep[inner] + 1) and np.all(dep[r] == dep[inner] + 1)
    # leaf boxes tight, inner boxes = union of the children (hence tight)
    lv = np.flatnonzero(leaf)
    ls = start[lv]
    assert np.all(np.diff(ls) > 0)
    assert np.array_equal(t["lo"][lv], np.minimum.reduceat(P, ls, axis=0)), "leaf box lo not tight"
    assert np.array_equal(t["hi"][lv], np.maximum.reduceat(P, ls, axis=0)), "leaf box hi not tight"
    assert np.array_equal(t["lo"][inner], np.minimum(t["lo"][l], t["lo"][r]))
    assert np.array_equal(t["hi"][inner], np.maximum(t["hi"][l], t["hi"][r]))
    # stability inside leaves
    steps = np.diff(perm)
    boundary = np.zeros(n - 1, bool) if n > 1 else np.zeros(0, bool)
    if n > 1:
        boundary[ls[1:] - 1] = True
        assert np.all((steps > 0) | boundary), "leaf not in stable order"
    # sides of every split, one depth at a time
    idx = np.flatnonzero(~leaf & ~np.asarray(t["index_split"], bool))
    pos = np.arange(n)
    for D in np.unique(dep[idx]):
        nd = idx[dep[idx] == D]
        nd = nd[np.argsort(start[nd])]
        owner = np.searchsorted(start[nd], pos, side="right") - 1
        ok = owner >= 0
        o = nd[np.clip(owner, 0, None)]
        ok &= pos < start[o] + count[o]
        o, p = o[ok], pos[ok]
        is_left = p < start[o] + count[left[o]]
        x = P[p, t["dim"][o]]
        s = np.asarray(t["split"], np.float32)[o]
        assert np.all((x < s) == is_left), f"a point is on the wrong side of a depth-{D} split"
    ix = np.flatnonzero(np.asarray(t["index_split"], bool) & ~leaf)
    assert np.array_equal(t["lo"][ix], t["hi"][ix]), "index split over non-identical points"


def assert_same_tree(a: dict, b: dict):
    """Node-by-node structural equality of two canonical trees."""
    assert len(a["leaf"]) == len(b["leaf"]), (len(a["leaf"]), len(b["leaf"]))
    for key in ("leaf", "index_split", "start", "count", "left", "right", "depth"):
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key
    inner = ~np.asarray(a["leaf"], bool)
    assert np.array_equal(np.asarray(a["dim"])[inner], np.asarray(b["dim"])[inner]), "dim"
    assert np.array_equal(np.asarray(a["split"])[inner], np.asarray(b["split"])[inner]), "split"
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"]), "boxes"
    assert np.array_equal(np.asarray(a["perm"]), np.asarray(b["perm"])), "leaf order"


def check_boxes(t: dict, points: np.ndarray):
    """Boxes of a tree whose points moved after the build (a refit): the leaf
    order is still a permutation, every leaf box is the exact box of its
    points, every inner box the union of its children's."""
    pts = np.asarray(points, np.float32)
    n = pts.shape[0]
    perm = np.asarray(t["perm"], np.int64)
    assert perm.shape == (n,) and np.all(np.bincount(perm, minlength=n) == 1)
    P = pts[perm]
    leaf = np.asarray(t["leaf"], bool)
    start = np.asarray(t["start"])
    lv = np.flatnonzero(leaf)
    ls = np.sort(start[lv])
    order = lv[np.argsort(start[lv])]
    assert np.array_equal(t["lo"][order], np.minimum.reduceat(P, ls, axis=0)), "leaf box lo not tight"
    assert np.array_equal(t["hi"][order], np.maximum.reduceat(P, ls, axis=0)), "leaf box hi not tight"
    inner = np.flatnonzero(~leaf)
    l, r = np.asarray(t["left"])[inner], np.asarray(t["right"])[inner]
    assert np.array_equal(t["lo"][inner], np.minimum(t["lo"][l], t["lo"][r]))
    assert np.array_equal(t["hi"][inner], np.maximum(t["hi"][l], t["hi"][r]))

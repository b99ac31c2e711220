"""Pins for the CPU oracle: checks against things the paper and mathematics fix,
never against the oracle itself.

* exact arithmetic on a 2^-4-scaled integer lattice (every FP32 op exact), where
  the answer is a closed form computed here with integers;
* FP64 recomputation of every returned distance (relative error <= 1e-6) and
  FP64 exhaustive search for the neighbour sets;
* hand-worked golden fixtures (tests/golden/);
* kd-tree invariants (permutation, ancestor sides, leaf <= B, tight boxes,
  stability, balance) and the split rules of Sec. III-A1 recomputed with numpy;
* special cases: a single bucket, k = n (full sort), k > n padding, 1-D windows,
  self queries.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1607_08220_gb300 import workloads
from tests import treecheck

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_lattice_knn(pts, q, k, scale_log2=4):
    """Closed form on lattice data: integer squared distances, order by (d2, id)."""
    P = np.rint(pts.astype(np.float64) * 2 ** scale_log2).astype(np.int64)
    Q = np.rint(q.astype(np.float64) * 2 ** scale_log2).astype(np.int64)
    n = P.shape[0]
    ids = np.full((Q.shape[0], k), -1, np.int64)
    d2 = np.full((Q.shape[0], k), np.inf, np.float64)
    for i in range(Q.shape[0]):
        di = ((P - Q[i]) ** 2).sum(axis=1)
        order = np.lexsort((np.arange(n), di))[:k]
        ids[i, :order.size] = order
        d2[i, :order.size] = di[order] / float(4 ** scale_log2)
    return ids, d2


# ----------------------------------------------------------------- brute force


@pytest.mark.parametrize("d", [1, 2, 3, 7])
def test_brute_exact_on_lattice(oracle_mod, d):
    pts = workloads.lattice_points(700, d, seed=10 + d, side=8)
    q = workloads.lattice_points(60, d, seed=20 + d, side=8)
    k = 17
    ids, d2 = oracle_mod.brute_knn(pts, q, k)
    eids, ed2 = exact_lattice_knn(pts, q, k)
    assert np.array_equal(ids, eids)
    assert np.array_equal(d2.astype(np.float64), ed2)


@pytest.mark.parametrize("d", [2, 3, 10])
def test_brute_fp64_recompute(oracle_mod, d):
    rng = np.random.default_rng(d)
    pts = rng.standard_normal((3000, d)).astype(np.float32)
    q = rng.standard_normal((80, d)).astype(np.float32)
    k = 12
    ids, d2 = oracle_mod.brute_knn(pts, q, k)
    P, Q = pts.astype(np.float64), q.astype(np.float64)
    for i in range(q.shape[0]):
        full = ((P - Q[i]) ** 2).sum(axis=1)
        exact = full[ids[i]]
        assert np.all(np.abs(d2[i] - exact) <= 1e-6 * exact + 1e-30)
        # the k returned points are the k nearest up to FP32 rounding
        kth = np.sort(full)[k - 1]
        assert np.all(exact <= kth * (1 + 2e-6) + 1e-30)
        assert np.all(np.diff(d2[i]) >= 0)


def test_brute_k_greater_than_n_pads(oracle_mod):
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]], np.float32)
    ids, d2 = oracle_mod.brute_knn(pts, np.zeros((1, 2), np.float32), 5)
    assert ids.tolist() == [[0, 1, 2, -1, -1]]
    assert d2[0, :3].tolist() == [0.0, 1.0, 4.0] and np.all(np.isinf(d2[0, 3:]))


def test_fp32_contract_no_fma(oracle_mod):
    """FP contract: each sub, mul and add is rounded on its own, dims in order.

    With q = (1 + 2^-12, sqrt(3) 2^-12) and x = 0 the unfused sum and a fused
    multiply-add on the second dimension (which keeps the exact square) round
    to different FP32 values; the oracle must give the unfused one.  The fused
    value is computed here with exact rationals."""
    from fractions import Fraction
    a = np.float32(1.0 + 2.0 ** -12)
    b = np.float32(math.sqrt(3.0) * 2.0 ** -12)
    pts = np.array([[0.0, 0.0]], np.float32)
    q = np.array([[a, b]], np.float32)
    ids, d2 = oracle_mod.brute_knn(pts, q, 1)
    t0 = np.float32(a * a)                         # exact a^2 has a tie bit below the ulp
    assert t0 == np.float32(1.0 + 2.0 ** -11)
    unfused = np.float32(t0 + np.float32(b * b))
    fused = np.float32(float(Fraction(float(t0)) + Fraction(float(b)) ** 2))
    assert unfused != fused
    assert d2[0, 0] == unfused


# ----------------------------------------------------------------- golden


@pytest.mark.parametrize("name", ["tiny_2d.json", "duplicates_1d.json"])
def test_golden_fixture(oracle_mod, name):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    pts = np.array(g["points"], np.float32)
    t = oracle_mod.build(pts, g["bucket"])
    e = t.export()
    assert e["perm"].tolist() == g["perm"]
    assert t.num_nodes == len(g["tree_preorder"])
    for i, nd in enumerate(g["tree_preorder"]):
        assert bool(e["leaf"][i]) == bool(nd["leaf"]), i
        assert e["start"][i] == nd["start"] and e["count"][i] == nd["count"], i
        assert e["depth"][i] == nd["depth"], i
        assert e["lo"][i].tolist() == nd["lo"] and e["hi"][i].tolist() == nd["hi"], i
        if not nd["leaf"]:
            assert bool(e["index_split"][i]) == bool(nd["index_split"]), i
            if not nd["index_split"]:
                assert e["dim"][i] == nd["dim"] and e["split"][i] == nd["split"], i
    for qi, (qq, k) in enumerate(zip(g["queries"], g["k"])):
        ids, d2 = oracle_mod.knn(t, np.array([qq], np.float32), k)
        assert ids[0].tolist() == g["ids"][qi]
        assert d2[0].tolist() == g["d2"][qi]
        bi, bd = oracle_mod.brute_knn(pts, np.array([qq], np.float32), k)
        assert bi[0].tolist() == g["ids"][qi] and bd[0].tolist() == g["d2"][qi]


# ----------------------------------------------------------------- tree


def _tree_cases():
    rng = np.random.default_rng(123)
    yield "uniform3", rng.random((20000, 3), dtype=np.float32), 32
    yield "cosmo3", workloads.cosmology_points(30000, seed=4, halos=8), 16
    yield "gauss10", rng.standard_normal((6000, 10)).astype(np.float32), 32
    yield "lattice2", workloads.lattice_points(5000, 2, seed=3, side=6), 8
    x = rng.random((3000, 3), dtype=np.float32)
    x[:, 1] = 0.25                                   # a constant dimension
    yield "constdim", x, 4
    y = np.repeat(rng.random((5, 2), dtype=np.float32), 400, axis=0)   # heavy duplicates
    yield "dups", y, 32
    yield "identical", np.full((300, 3), 0.5, np.float32), 8
    z = np.zeros((2048, 1), np.float32)
    z[1::2] = 0.7
    z[0::2] = 0.1
    yield "sample_all_min", z, 1024                  # every sample equals the node minimum


@pytest.mark.parametrize("case", list(_tree_cases()), ids=lambda c: c[0])
def test_tree_invariants(oracle_mod, case):
    name, pts, B = case
    t = oracle_mod.build(pts, B)
    e = t.export()
    treecheck.check_invariants(e, pts, B)
    if name in ("uniform3", "cosmo3", "gauss10"):
        assert t.depth <= treecheck.balance_bound(pts.shape[0], B)
    checked = 0
    for i in np.flatnonzero(~e["leaf"] & ~e["index_split"]):
        if treecheck.check_split_dim(e, pts, int(i)):
            treecheck.check_split_rule(e, pts, int(i))
            checked += 1
    if name in ("uniform3", "cosmo3", "gauss10", "lattice2"):
        assert checked > 0


def test_sample_all_min_fallback(oracle_mod):
    """Samples all at the node minimum: the split falls back to the next larger value."""
    z = np.zeros((2048, 1), np.float32)
    z[1::2] = 0.7
    z[0::2] = 0.1
    e = oracle_mod.build(z, 1024).export()
    assert not e["leaf"][0] and not e["index_split"][0]
    assert e["split"][0] == np.float32(0.7) and e["count"][1] == 1024


def test_exact_median_small_nodes(oracle_mod):
    """With n_node <= 1024 every point is a sample: the split is an exact median."""
    rng = np.random.default_rng(5)
    pts = rng.permutation(1000).astype(np.float32)[:, None]
    e = oracle_mod.build(pts, 10).export()
    assert e["split"][0] == 500.0 and e["count"][1] == 500


def test_depth_paper_scale_balance(oracle_mod):
    """Near-balanced tree (the paper reports depth 21 for 50M points at B=32,
    i.e. ceil(log2(n/B))): depth stays within 2 of that on clustered data."""
    pts = workloads.cosmology_points(1 << 18, seed=0, halos=64)
    t = oracle_mod.build(pts, 32)
    assert t.depth <= treecheck.balance_bound(pts.shape[0], 32)


# ----------------------------------------------------------------- Algorithm 1


def _knn_cases():
    rng = np.random.default_rng(7)
    for d in (1, 2, 3, 5, 10, 16):
        for n in (1, 2, 7, 33, 500, 2500):
            pts = rng.standard_normal((n, d)).astype(np.float32)
            q = rng.standard_normal((40, d)).astype(np.float32)
            for k in (1, 5, 32):
                yield f"gauss_d{d}_n{n}_k{k}", pts, q, k, 4 if n < 100 else 32
    lat = workloads.lattice_points(3000, 3, seed=1, side=5)
    yield "lattice_ties", lat, workloads.lattice_points(100, 3, seed=2, side=5), 20, 16
    yield "lattice_k_eq_n", lat[:200], lat[:30], 200, 8
    yield "single_bucket", lat[:30], lat[:10], 7, 32
    dup = np.repeat(rng.random((7, 3), dtype=np.float32), 50, axis=0)
    yield "duplicates", dup, dup[::13], 60, 8


@pytest.mark.parametrize("case", list(_knn_cases()), ids=lambda c: c[0])
def test_tree_knn_equals_brute(oracle_mod, case):
    name, pts, q, k, B = case
    t = oracle_mod.build(pts, B)
    ids, d2 = oracle_mod.knn(t, q, k)
    bi, bd = oracle_mod.brute_knn(pts, q, k)
    assert np.array_equal(ids, bi)
    assert np.array_equal(d2.view(np.uint32), bd.view(np.uint32))


def test_tree_knn_lattice_closed_form(oracle_mod):
    pts = workloads.lattice_points(4000, 3, seed=11, side=9)
    q = workloads.lattice_points(200, 3, seed=12, side=9)
    t = oracle_mod.build(pts, 32)
    ids, d2 = oracle_mod.knn(t, q, 25)
    eids, ed2 = exact_lattice_knn(pts, q, 25)
    assert np.array_equal(ids, eids) and np.array_equal(d2.astype(np.float64), ed2)


def test_one_dimensional_window(oracle_mod):
    """In 1-D the k nearest of a query form a contiguous run of the sorted points."""
    rng = np.random.default_rng(2)
    x = rng.permutation(5000).astype(np.float32)[:, None] * np.float32(0.5)
    q = (rng.random((200, 1)) * 2500).astype(np.float32)
    t = oracle_mod.build(x, 16)
    ids, _ = oracle_mod.knn(t, q, 9)
    rank = np.argsort(np.argsort(x[:, 0]))
    for row in ids:
        r = np.sort(rank[row])
        assert r[-1] - r[0] == 8


def test_self_query_rank0(oracle_mod):
    rng = np.random.default_rng(3)
    pts = rng.random((5000, 3), dtype=np.float32)
    t = oracle_mod.build(pts, 32)
    ids, d2 = oracle_mod.knn(t, pts, 1)
    assert np.array_equal(ids[:, 0], np.arange(5000)) and np.all(d2[:, 0] == 0)


def test_literal_bound_over_prunes(oracle_mod):
    """Reading C1, built through the oracle: 1-D points whose tree splits
    dimension 0 twice on the way to the bucket holding 2.1 (root at s = 1.0,
    then s = 2.1).  For q = 0 and k = 6, Algorithm 1's accumulated bound for
    that bucket is sqrt(1.0^2 + 2.1^2) > 2.2, the 6th distance once the other
    buckets are scanned (the point -2.2), so the literal algorithm would prune
    it and return -2.2 as the 6th neighbour; the true 6th neighbour is 2.1
    (distance 2.1 < 2.2).  The oracle's tight-box bound (2.1^2) must visit it."""
    x = np.array([[-2.2], [-0.5], [0.2], [0.5], [1.0], [1.5], [2.1], [2.5]], np.float32)
    t = oracle_mod.build(x, 2)
    e = t.export()
    # preorder: root, left subtree (3 nodes), right child, its two leaves
    assert e["split"][0] == np.float32(1.0) and e["dim"][0] == 0
    right = int(e["right"][0])
    assert e["split"][right] == np.float32(2.1) and e["dim"][right] == 0
    far = int(e["right"][right])
    assert e["leaf"][far] and sorted(e["perm"][e["start"][far]:e["start"][far] + e["count"][far]]) == [6, 7]
    literal = math.sqrt(float(np.float32(1.0)) ** 2 + float(np.float32(2.1)) ** 2)
    sixth_without = abs(float(np.float32(-2.2)))
    assert literal > sixth_without > abs(float(np.float32(2.1)))
    ids, d2 = oracle_mod.knn(t, np.zeros((1, 1), np.float32), 6)
    assert ids[0].tolist() == [2, 1, 3, 4, 5, 6]          # 0.2, -0.5, 0.5, 1.0, 1.5, 2.1
    assert d2[0, 5] == np.float32(np.float32(2.1) * np.float32(2.1))
    bi, bd = oracle_mod.brute_knn(x, np.zeros((1, 1), np.float32), 6)
    assert np.array_equal(ids, bi) and np.array_equal(d2.view(np.uint32), bd.view(np.uint32))


# ------------------------------------------------------------------ reading R2 (summation order)


def _variance_nodes():
    with open(os.path.join(GOLDEN, "variance_order.json")) as f:
        return json.load(f)["nodes"]


def _root_choice(oracle_mod, node, lib=None):
    pts = np.array(node["points"], np.float32)
    e = oracle_mod.build(pts, node["bucket"], lib=lib).export()
    return int(e["dim"][0]), e


@pytest.mark.parametrize("node", _variance_nodes(), ids=lambda n: n["name"])
def test_variance_order_golden(oracle_mod, node):
    """Hand-worked nodes (tests/golden/variance_order.json) whose split
    dimension depends on the exact FP32 summation order of reading R2."""
    dim, e = _root_choice(oracle_mod, node)
    assert not e["leaf"][0] and not e["index_split"][0]
    assert dim == node["dim"]
    assert e["split"][0] == np.float32(node["split"])
    assert e["count"][1] == node["left_count"] and e["leaf"][1] and e["leaf"][2]
    assert e["perm"].tolist() == node["perm"]
    assert e["lo"].tolist() == node["lo"] and e["hi"].tolist() == node["hi"]


# Planted mistakes: the body of the oracle's fixed-order sum replaced by a
# plausible other order; each must change a golden node's split dimension.
_SUM_BODY = """    float part[32];
    for (int p = 0; p < 32; p++) part[p] = 0.0f;
    for (int64_t j = 0; j < cnt; j++) part[j % 32] = part[j % 32] + vals[j];
    for (int off = 16; off >= 1; off /= 2)
        for (int p = 0; p < off; p++) part[p] = part[p] + part[p + off];
    return part[0];"""
_MUTANTS = {
    "sequential": ("""    float acc = 0.0f;
    for (int64_t j = 0; j < cnt; j++) acc = acc + vals[j];
    return acc;""", "A_strided_vs_sequential"),
    "fp64": ("""    double acc = 0.0;
    for (int64_t j = 0; j < cnt; j++) acc = acc + (double)vals[j];
    return (float)acc;""", "B_ties_vs_exact"),
    "partials_in_sequence": ("""    float part[32];
    for (int p = 0; p < 32; p++) part[p] = 0.0f;
    for (int64_t j = 0; j < cnt; j++) part[j % 32] = part[j % 32] + vals[j];
    float acc = 0.0f;
    for (int p = 0; p < 32; p++) acc = acc + part[p];
    return acc;""", "A_strided_vs_sequential"),
}


@pytest.mark.parametrize("mutant", sorted(_MUTANTS))
def test_variance_order_catches_planted_mistakes(oracle_mod, mutant):
    src = oracle_mod.source_text()
    assert src.count(_SUM_BODY) == 1, "the oracle's fixed-order sum changed: update this test"
    body, catcher = _MUTANTS[mutant]
    lib = oracle_mod.compile_variant(src.replace(_SUM_BODY, body), mutant)
    nodes = {n["name"]: n for n in _variance_nodes()}
    dim, _ = _root_choice(oracle_mod, nodes[catcher], lib=lib)
    assert dim != nodes[catcher]["dim"], f"a {mutant} sum was not caught by {catcher}"


# ------------------------------------------------------------------ radius-bounded KNN (Algorithm 1's r)


def _numpy_radius_knn(pts, q, k, r2):
    """The plain definition written with numpy FP32 elementwise ops (each op
    rounded, dims in order, no FMA): the k smallest (d2, id) among d2 <= r2."""
    pts = pts.astype(np.float32)
    out_i = np.full((q.shape[0], k), -1, np.int32)
    out_d = np.full((q.shape[0], k), np.inf, np.float32)
    for r in range(q.shape[0]):
        diff = (q[r][None, :] - pts).astype(np.float32)
        sq = (diff * diff).astype(np.float32)
        d2 = sq[:, 0].copy()
        for j in range(1, pts.shape[1]):
            d2 = (d2 + sq[:, j]).astype(np.float32)
        ok = np.flatnonzero(d2 <= np.float32(r2))
        order = ok[np.lexsort((ok, d2[ok]))][:k]
        out_i[r, :order.size] = order
        out_d[r, :order.size] = d2[order]
    return out_i, out_d


def test_radius_brute_matches_numpy_definition(oracle_mod):
    rng = np.random.default_rng(31)
    pts = rng.random((700, 3), dtype=np.float32)
    q = rng.random((60, 3), dtype=np.float32)
    for r2 in (0.0, 0.001, 0.01, 0.05, np.inf):
        bi, bd = oracle_mod.brute_knn(pts, q, 9, max_d2=r2)
        ni, nd = _numpy_radius_knn(pts, q, 9, r2)
        assert np.array_equal(bi, ni) and np.array_equal(bd.view(np.uint32), nd.view(np.uint32))


def test_radius_tree_matches_brute_with_ties_on_the_radius(oracle_mod):
    # lattice points: many distances equal the radius exactly (inclusive bound)
    pts = workloads.lattice_points(3000, 3, seed=8, side=8)
    q = workloads.lattice_points(200, 3, seed=9, side=8)
    t = oracle_mod.build(pts, 8)
    for r2 in (0.0, 2.0 ** -8, 3 * 2.0 ** -8, 2.0 ** -4, 1.0):
        ti, td = oracle_mod.knn(t, q, 12, max_d2=r2)
        bi, bd = oracle_mod.brute_knn(pts, q, 12, max_d2=r2)
        assert np.array_equal(ti, bi) and np.array_equal(td.view(np.uint32), bd.view(np.uint32))
        assert np.all((td <= np.float32(r2)) | (ti == -1))


def test_radius_special_cases(oracle_mod):
    rng = np.random.default_rng(32)
    pts = rng.random((500, 2), dtype=np.float32)
    pts[10] = pts[3]                                   # one exact duplicate pair
    t = oracle_mod.build(pts, 4)
    # r2 = 0: a self query finds only itself and its exact duplicates
    ti, td = oracle_mod.knn(t, pts, 3, max_d2=0.0)
    assert np.array_equal(ti[:, 0][np.arange(500) != 10], np.arange(500)[np.arange(500) != 10])
    assert ti[3].tolist()[:2] == [3, 10] and ti[10].tolist()[:2] == [3, 10]
    assert (ti[:, 2] == -1).all() and np.isinf(td[:, 2]).all()
    # r2 = +inf is the unbounded query
    ui, ud = oracle_mod.knn(t, pts, 5)
    ri, rd = oracle_mod.knn(t, pts, 5, max_d2=np.inf)
    assert np.array_equal(ui, ri) and np.array_equal(ud.view(np.uint32), rd.view(np.uint32))

"""Batched form (many independent sets in one graph launch): every set's
neighbours and distances equal, bit for bit, those of building and querying
that set on its own (panda_build + panda_knn), which the single-tree parity
tests tie to the oracle; a few sets are also checked against the oracle
directly.  Graph replays with new inputs must stay exact."""
import numpy as np
import pytest

import oracle
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


def make_sets(seed, nsets, lo, hi, d=3, kchoices=(4, 8, 16, 32)):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), nsets))).astype(np.int64)
    sets = []
    for i, n in enumerate(sizes):
        n = int(n)
        if d == 3:
            pts = workloads.cosmology_points(n, seed=seed * 1000 + i, halos=max(1, n // 5000))
            q = workloads.cosmology_points(max(0, n // 10), seed=seed * 1000 + 500 + i, halos=max(1, n // 5000))
        else:
            pts = rng.standard_normal((n, d)).astype(np.float32)
            q = rng.standard_normal((max(0, n // 10), d)).astype(np.float32)
        sets.append((pts, q, int(rng.choice(kchoices))))
    return sets


def fill(batch, sets):
    import torch
    for s, (pts, q, k) in enumerate(sets):
        a, b = batch.point_off[s], batch.point_off[s + 1]
        batch.points[a:b].copy_(torch.from_numpy(pts))
        a, b = batch.query_off[s], batch.query_off[s + 1]
        if b > a:
            batch.queries[a:b].copy_(torch.from_numpy(q))


def check_against_single(P, batch, sets, oracle_sets=()):
    import torch
    for s, (pts, q, k) in enumerate(sets):
        if q.shape[0] == 0:
            continue
        ids, d2 = batch.result(s)
        t = P.build(torch.from_numpy(pts).cuda(), 32)
        ri, rd = P.knn(t, torch.from_numpy(q).cuda(), k)
        torch.cuda.synchronize()
        assert torch.equal(ids, ri), f"set {s}: ids differ"
        assert torch.equal(d2.view(torch.int32), rd.view(torch.int32)), f"set {s}: d2 differ"
        if s in oracle_sets:
            ot = oracle.build(pts, 32)
            ei, ed = oracle.knn(ot, q, k)
            assert np.array_equal(ids.cpu().numpy(), ei)
            assert np.array_equal(d2.cpu().numpy().view(np.uint32), ed.view(np.uint32))


def test_batch_matches_single_trees_and_replays(P):
    import torch
    sets = make_sets(31, 40, 50, 120_000)
    sets[3] = (sets[3][0][:3], sets[3][1][:5], 16)          # fewer points than k: padding
    sets[7] = (sets[7][0][:1], sets[7][1][:0], 4)           # one point, no queries
    batch = P.Batch([p.shape[0] for p, _, _ in sets], [q.shape[0] for _, q, _ in sets],
                    [k for _, _, k in sets], d=3, bucket=32)
    fill(batch, sets)
    batch.run()
    torch.cuda.synchronize()
    batch.status()
    check_against_single(P, batch, sets, oracle_sets=(0, 3, 11))
    info = batch.info()
    assert info["kernels_per_run"] > 10
    # replay the captured graph with new inputs of the same sizes
    sets2 = [(np.random.default_rng(100 + i).random(p.shape, dtype=np.float32),
              np.random.default_rng(200 + i).random(q.shape, dtype=np.float32), k)
             for i, (p, q, k) in enumerate(sets)]
    fill(batch, sets2)
    batch.run()
    torch.cuda.synchronize()
    batch.status()
    check_against_single(P, batch, sets2, oracle_sets=(1,))
    # every set forced to each traversal shape: still exact (replays the same graph)
    for trav in ("packet", "per_query"):
        batch.set_query_params(0, trav)
        batch.run()
        torch.cuda.synchronize()
        batch.status()
        check_against_single(P, batch, sets2)
    batch.free()


def test_batch_ten_dims(P):
    import torch
    sets = make_sets(7, 12, 200, 40_000, d=10, kchoices=(1, 10, 16))
    batch = P.Batch([p.shape[0] for p, _, _ in sets], [q.shape[0] for _, q, _ in sets],
                    [k for _, _, k in sets], d=10, bucket=32)
    fill(batch, sets)
    batch.run()
    torch.cuda.synchronize()
    batch.status()
    check_against_single(P, batch, sets, oracle_sets=(2,))
    batch.free()


def test_batch_nonfinite_reported(P):
    import torch
    sets = make_sets(3, 4, 100, 2000)
    p0 = sets[0][0].copy()
    p0[5, 1] = np.nan
    sets[0] = (p0, sets[0][1], sets[0][2])
    batch = P.Batch([p.shape[0] for p, _, _ in sets], [q.shape[0] for _, q, _ in sets],
                    [k for _, _, k in sets], d=3)
    fill(batch, sets)
    batch.run()
    torch.cuda.synchronize()
    with pytest.raises(P.PandaError) as e:
        batch.status()
    assert e.value.status == 2
    batch.free()

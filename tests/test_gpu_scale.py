"""Oracle parity of the batched and served forms at the benchmark's full sizes.

* Batched form, 512 independent sets (sizes log-uniform in [1e3, 2e6],
  cosmology-like, 10% queries each, k in {4, 8, 16, 32}), built and queried
  by one captured graph with the autotuned bucket size: every set's sampled
  rows against the oracle's exhaustive search, and five sets (the smallest,
  the quartiles, the largest) in full against the oracle's Algorithm 1.
* Served form on the plasma-like slab: a resident tree of 1e8 points, the
  Poisson request stream of one second (about 2,000 requests, sizes
  log-uniform in [1, 1e6], k in {1, 8, 32}) and a second tree of 2e7 points
  admitted while requests run.  At least 1,000 sampled rows per tree against
  the oracle's exhaustive search (ids bit-exact, distances to 0 ULP), and
  every request equal to panda_knn on its own tree (the same alone and in the
  mix).
"""
import concurrent.futures as cf
import threading

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
    oracle.compile_oracle()
    return panda


def assert_rows(gi, gd, ei, ed, what):
    bad = np.flatnonzero((gi != ei).any(axis=1))
    assert bad.size == 0, f"{what}: {bad.size} rows differ from the oracle, first {bad[:5]}"
    assert np.array_equal(gd.view(np.uint32), ed.view(np.uint32)), f"{what}: d2 differ from the oracle"


def test_batched_512_sets_against_oracle(P):
    import torch
    sets = workloads.batched_sets(nsets=512)
    npts = [p.shape[0] for p, _, _ in sets]
    nq = [q.shape[0] for _, q, _ in sets]
    ks = [k for _, _, k in sets]
    big = int(np.argmax(npts))
    tuned = P.tune(torch.from_numpy(sets[big][0]).cuda(), torch.from_numpy(sets[big][1]).cuda(),
                   k=ks[big], m_total=nq[big])
    batch = P.Batch(npts, nq, ks, d=3, bucket=tuned["bucket"])
    batch.set_query_params(tuned["transpose_max"], tuned["traversal"])
    for s, (pts, q, k) in enumerate(sets):
        batch.points[batch.point_off[s]:batch.point_off[s + 1]].copy_(torch.from_numpy(pts))
        batch.queries[batch.query_off[s]:batch.query_off[s + 1]].copy_(torch.from_numpy(q))
    for _ in range(2):          # the capture, then a replay of the graph
        batch.run()
        torch.cuda.synchronize()
        batch.status()
    results = [tuple(x.cpu().numpy() for x in batch.result(s)) for s in range(len(sets))]
    batch.free()
    rng = np.random.default_rng(512)
    picks = [np.sort(rng.choice(q.shape[0], min(q.shape[0], 16), replace=False)) for _, q, _ in sets]

    def sampled(s):
        pts, q, k = sets[s]
        rows = picks[s]
        bi, bd = oracle.brute_knn(pts, q, k, rows=rows, threads=1)
        gi, gd = results[s]
        assert_rows(gi[rows], gd[rows], bi, bd, f"set {s} (n={pts.shape[0]})")
        return rows.size

    order = np.argsort(npts)
    full = sorted({int(order[int(f * (len(sets) - 1))]) for f in (0.0, 0.25, 0.5, 0.75, 1.0)})

    def complete(s):
        pts, q, k = sets[s]
        ei, ed = oracle.knn(oracle.build(pts, tuned["bucket"]), q, k, threads=1)
        assert_rows(*results[s], ei, ed, f"set {s} (n={pts.shape[0]}, full)")
        return q.shape[0]

    with cf.ThreadPoolExecutor(16) as ex:        # the oracle's C calls release the GIL
        checked = sum(ex.map(sampled, range(len(sets))))
        checked_full = sum(ex.map(complete, full))
    assert checked >= 512 * 10 and checked_full > 100_000


def test_served_plasma_100m_with_second_tree(P):
    import torch
    pts0 = workloads.plasma_points(100_000_000, seed=0)
    pts1 = workloads.plasma_points(20_000_000, seed=4)
    reqs = workloads.plasma_requests(duration_s=1.0)
    qs = [workloads.plasma_points(r["m"], seed=r["seed"]) for r in reqs]
    dev0, dev1 = torch.from_numpy(pts0).cuda(), torch.from_numpy(pts1).cuda()
    qdev = [torch.from_numpy(q).cuda() for q in qs]
    outs = [(torch.empty((r["m"], r["k"]), dtype=torch.int32, device="cuda"),
             torch.empty((r["m"], r["k"]), dtype=torch.float32, device="cuda")) for r in reqs]
    torch.cuda.synchronize()
    srv = P.Server()
    tree_ids = [srv.add_tree(dev0)]
    admitted = threading.Event()

    def admit():
        tree_ids.append(srv.add_tree(dev1))
        admitted.set()

    admitter = None
    rids = []
    for i, r in enumerate(reqs):
        if admitter is None and r["t"] >= 0.5:      # the second tree arrives mid-stream
            admitter = threading.Thread(target=admit)
            admitter.start()
        if r["tree"] == 1:
            admitted.wait()
        rids.append(srv.submit(tree_ids[r["tree"]], qdev[i], r["k"], outs[i]))
    for rid in rids:
        srv.wait(rid, 600)
    admitter.join()
    st = srv.stats()
    assert st["batches"] < len(reqs)                 # requests were coalesced
    srv.close()
    # each request alone (panda_knn on its own tree) equals its row in the mix
    plain = [P.build(dev0, 32), P.build(dev1, 32)]
    for i, r in enumerate(reqs):
        ri, rd = P.knn(plain[r["tree"]], qdev[i], r["k"])
        torch.cuda.synchronize()
        assert torch.equal(outs[i][0], ri) and torch.equal(outs[i][1].view(torch.int32), rd.view(torch.int32)), i
    for t in plain:
        t.free()
    # >= 1,000 sampled rows per tree against exhaustive search
    rng = np.random.default_rng(3)
    for tree, pts in ((0, pts0), (1, pts1)):
        mine = [i for i, r in enumerate(reqs) if r["tree"] == tree]
        sizes = np.array([reqs[i]["m"] for i in mine])
        picks = np.sort(rng.choice(int(sizes.sum()), 1200, replace=False))
        cum = np.concatenate([[0], np.cumsum(sizes)])
        owner = np.searchsorted(cum, picks, side="right") - 1
        q_rows, got = [], []
        for j in np.unique(owner):
            i = mine[j]
            rows = picks[owner == j] - cum[j]
            q_rows.append(qs[i][rows])
            ri = torch.from_numpy(rows).cuda()
            got.append((i, outs[i][0][ri].cpu().numpy(), outs[i][1][ri].cpu().numpy()))
        bi, bd = oracle.brute_knn(pts, np.concatenate(q_rows), 32)
        at = 0
        for i, gi, gd in got:
            k, c = reqs[i]["k"], gi.shape[0]
            # the k nearest are the first k of the 32 nearest (keys are unique)
            assert_rows(gi, gd, bi[at:at + c, :k], np.ascontiguousarray(bd[at:at + c, :k]),
                        f"tree {tree} request {i}")
            at += c
        assert at == 1200

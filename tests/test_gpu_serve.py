"""Served form: requests of different trees, sizes and k coalesced into shared
launches return exactly the CPU oracle's answer for their own tree (ids
bit-exact, distances to 0 ULP) and exactly what each request returns alone
(panda_knn on the same tree); a tree can be admitted while requests run, and
admission respects the memory budget."""
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
    return panda


def alone(P, tree, q, k):
    import torch
    ids, d2 = P.knn(tree, q, k)
    torch.cuda.synchronize()
    return ids, d2


def assert_oracle(otree, q_np, out):
    """The served rows against the oracle's Algorithm 1 on the same points."""
    import torch
    torch.cuda.synchronize()
    ei, ed = oracle.knn(otree, q_np, out[0].shape[1])
    gi, gd = out[0].cpu().numpy(), out[1].cpu().numpy()
    bad = np.flatnonzero((gi != ei).any(axis=1))
    assert bad.size == 0, f"{bad.size} rows differ from the oracle, first {bad[:5]}"
    assert np.array_equal(gd.view(np.uint32), ed.view(np.uint32)), "d2 differ from the oracle"


def test_mixed_requests_equal_alone(P):
    import torch
    rng = np.random.default_rng(5)
    np_a = workloads.cosmology_points(200_000, seed=50, halos=30)
    np_b = workloads.plasma_points(150_000, seed=51)
    np_c = workloads.cosmology_points(30_000, seed=52, halos=5)
    otrees = [oracle.build(x, 32) for x in (np_a, np_b, np_c)]
    pts_a, pts_b, pts_c = (torch.from_numpy(x).cuda() for x in (np_a, np_b, np_c))
    srv = P.Server(max_batch_queries=40_000)
    tids = [srv.add_tree(pts_a), srv.add_tree(pts_b), srv.add_tree(pts_c)]
    refs = [P.build(pts_a, 32), P.build(pts_b, 32), P.build(pts_c, 32)]
    todo = []
    for i in range(90):
        # requests of the small tree c are often dense (more than n/4 queries:
        # packet traversal), the others sparse (a lane per query)
        tree = int(rng.integers(0, 3))
        m = int(np.floor(np.exp(rng.uniform(0, np.log(20_001)))))
        k = int(rng.choice([1, 8, 32]))
        q = (workloads.plasma_points(m, seed=1000 + i) if tree == 1
             else workloads.cosmology_points(m, seed=1000 + i, halos=30 if tree == 0 else 5))
        qd = torch.from_numpy(q).cuda()
        out = (torch.empty((m, k), dtype=torch.int32, device="cuda"),
               torch.empty((m, k), dtype=torch.float32, device="cuda"))
        todo.append((tree, q, qd, k, out))
    torch.cuda.synchronize()
    reqs = [(srv.submit(tids[tree], qd, k, out), tree, q, qd, k, out) for tree, q, qd, k, out in todo]
    for rid, tree, q, qd, k, out in reqs:
        srv.wait(rid, 60)
        assert_oracle(otrees[tree], q, out)
        ri, rd = alone(P, refs[tree], qd, k)
        assert torch.equal(out[0], ri)
        assert torch.equal(out[1].view(torch.int32), rd.view(torch.int32))
    st = srv.stats()
    assert st["requests"] == 90 and st["batches"] < 90          # requests were coalesced
    batches = {srv.times(r[0])[2] for r in reqs}
    assert len(batches) == st["batches"]
    srv.close()


def test_tree_admitted_while_requests_run(P):
    import torch
    np_a = workloads.cosmology_points(300_000, seed=60, halos=40)
    np_b = workloads.cosmology_points(250_000, seed=61, halos=40)
    ot_a, ot_b = oracle.build(np_a, 32), oracle.build(np_b, 32)
    pts_a, pts_b = torch.from_numpy(np_a).cuda(), torch.from_numpy(np_b).cuda()
    srv = P.Server(max_batch_queries=1 << 20)
    ta = srv.add_tree(pts_a)
    ref_a, ref_b = P.build(pts_a, 32), P.build(pts_b, 32)
    result = {}

    def admit():
        result["tb"] = srv.add_tree(pts_b)

    th = threading.Thread(target=admit)
    reqs = []
    for i in range(30):
        if i == 5:
            th.start()
        q = workloads.cosmology_points(20_000, seed=2000 + i, halos=40)
        qd = torch.from_numpy(q).cuda()
        out = (torch.empty((20_000, 8), dtype=torch.int32, device="cuda"),
               torch.empty((20_000, 8), dtype=torch.float32, device="cuda"))
        reqs.append((srv.submit(ta, qd, 8, out), ref_a, ot_a, q, qd, out))
    th.join()
    q = workloads.cosmology_points(10_000, seed=3000, halos=40)
    qd = torch.from_numpy(q).cuda()
    out = (torch.empty((10_000, 5), dtype=torch.int32, device="cuda"),
           torch.empty((10_000, 5), dtype=torch.float32, device="cuda"))
    reqs.append((srv.submit(result["tb"], qd, 5, out), ref_b, ot_b, q, qd, out))
    for rid, ref, ot, q, qd, out in reqs:
        srv.wait(rid, 60)
        assert_oracle(ot, q, out)
        ri, rd = alone(P, ref, qd, out[0].shape[1])
        assert torch.equal(out[0], ri) and torch.equal(out[1].view(torch.int32), rd.view(torch.int32))
    srv.close()


def test_admission_budget_and_errors(P):
    import torch
    pts = torch.from_numpy(np.random.default_rng(0).random((100_000, 3), dtype=np.float32)).cuda()
    srv = P.Server(mem_budget_bytes=1 << 20)       # 1 MiB: a 100k-point tree does not fit
    with pytest.raises(P.PandaError) as e:
        srv.add_tree(pts)
    assert e.value.status == 4
    srv.close()
    srv = P.Server()
    t = srv.add_tree(pts)
    q = pts[:100]
    out = (torch.empty((100, 65), dtype=torch.int32, device="cuda"),
           torch.empty((100, 65), dtype=torch.float32, device="cuda"))
    with pytest.raises(P.PandaError) as e:
        srv.submit(t, q, 65, out)
    assert e.value.status == 3
    with pytest.raises(P.PandaError) as e:
        srv.submit(t + 7, q, 4, out)
    assert e.value.status == 1
    with pytest.raises(P.PandaError) as e:
        srv.wait(123456, 0.01)
    assert e.value.status == 1
    out = (torch.empty((100, 4), dtype=torch.int32, device="cuda"),
           torch.empty((100, 4), dtype=torch.float32, device="cuda"))
    rid = srv.submit(t, q, 4, out)
    srv.wait(rid, 30)
    assert torch.equal(out[0][:, 0].cpu(), torch.arange(100, dtype=torch.int32))
    srv.close()


def test_nonfinite_request_fails_alone(P):
    """A request holding a NaN query fails with PANDA_ERR_NONFINITE_INPUT; the
    requests batched with it still return panda_knn's answers."""
    import torch
    np_pts = workloads.cosmology_points(100_000, seed=80, halos=20)
    ot = oracle.build(np_pts, 32)
    pts = torch.from_numpy(np_pts).cuda()
    srv = P.Server()
    t = srv.add_tree(pts)
    ref = P.build(pts, 32)
    todo = []
    for i in range(12):
        qn = workloads.cosmology_points(3000, seed=900 + i, halos=20)
        q = torch.from_numpy(qn).cuda()
        if i == 5:
            q[17, 1] = float("nan")
        out = (torch.empty((3000, 4), dtype=torch.int32, device="cuda"),
               torch.empty((3000, 4), dtype=torch.float32, device="cuda"))
        todo.append((qn, q, out))
    torch.cuda.synchronize()
    rids = [srv.submit(t, q, 4, out) for _, q, out in todo]
    for i, (rid, (qn, q, out)) in enumerate(zip(rids, todo)):
        if i == 5:
            with pytest.raises(P.PandaError) as e:
                srv.wait(rid, 60)
            assert e.value.status == 2
            continue
        srv.wait(rid, 60)
        assert_oracle(ot, qn, out)
        ri, rd = alone(P, ref, q, 4)
        assert torch.equal(out[0], ri) and torch.equal(out[1].view(torch.int32), rd.view(torch.int32))
    srv.close()


def test_query_batches_wait_for_memory(P):
    """Admission of query batches by memory: with a budget that holds the tree
    and the scratch of one 50,000-query batch but not of two (about 1.2 MB
    against 2.5 MB), eight such requests submitted at once run one batch at a
    time -- the others wait in the queue -- and each equals the oracle's
    answer.  A request whose scratch can never fit fails with
    PANDA_ERR_OUT_OF_MEMORY instead of waiting forever; a submit beyond the
    queue limit is refused with PANDA_ERR_QUEUE_FULL."""
    import torch
    np_pts = workloads.cosmology_points(200_000, seed=81, halos=30)
    ot = oracle.build(np_pts, 32)
    pts = torch.from_numpy(np_pts).cuda()
    probe = P.Server()
    probe.add_tree(pts)
    tree_bytes = probe.stats()["bytes_used"]
    probe.close()
    srv = P.Server(mem_budget_bytes=tree_bytes + 1_800_000)
    t = srv.add_tree(pts)
    reqs = []
    for i in range(8):
        qn = workloads.cosmology_points(50_000, seed=1100 + i, halos=30)
        out = (torch.empty((50_000, 6), dtype=torch.int32, device="cuda"),
               torch.empty((50_000, 6), dtype=torch.float32, device="cuda"))
        reqs.append((qn, torch.from_numpy(qn).cuda(), out))
    torch.cuda.synchronize()
    rids = [srv.submit(t, qd, 6, out) for _, qd, out in reqs]
    for rid, (qn, _, out) in zip(rids, reqs):
        srv.wait(rid, 120)
        assert_oracle(ot, qn, out)
    adm = srv.admission()
    assert adm["deferred_requests"] >= 1 and adm["scratch_reserved"] == 0 and adm["pending_queries"] == 0
    assert srv.stats()["batches"] == 8                       # no two requests' scratch fit together
    big = torch.from_numpy(workloads.cosmology_points(200_000, seed=1200, halos=30)).cuda()
    out = (torch.empty((200_000, 6), dtype=torch.int32, device="cuda"),
           torch.empty((200_000, 6), dtype=torch.float32, device="cuda"))
    rid = srv.submit(t, big, 6, out)
    with pytest.raises(P.PandaError) as e:
        srv.wait(rid, 120)
    assert e.value.status == 4
    srv.set_queue_limit(60_000)
    with pytest.raises(P.PandaError) as e:
        srv.submit(t, big[:70_000], 6, (out[0][:70_000], out[1][:70_000]))
    assert e.value.status == 7
    qn, qd, out = reqs[0]
    rid = srv.submit(t, qd, 6, out)                          # within the limit: accepted and exact
    srv.wait(rid, 120)
    assert_oracle(ot, qn, out)
    srv.close()

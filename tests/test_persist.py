"""Tree checkpoint: a saved tree loads back and answers exactly as before; a
file that is not a saved tree, is truncated or holds ids that are not a
permutation is refused before anything reaches the device (the refusals run
on the CPU; the round trip needs a GPU)."""
import os
import struct

import numpy as np
import pytest

from paper_1607_08220_gb300 import workloads

MAGIC = b"PANDAKD1"


def _lib():
    from paper_1607_08220_gb300 import build_ext, panda
    build_ext.build()
    return panda


def _write(path, n, d, dp, nv, ns, slots, ids, nodes=None):
    hdr = [n, d, dp, 32, nv, ns, 1024, slots, slots, 1, 1, slots]
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<12q", *hdr))
        f.write(np.zeros(32, np.float32).tobytes())
        if nodes is None:
            nodes = np.zeros((slots, ns * 4), np.int32)
            nodes[0, :4] = [0, n, 0, np.int32(np.uint32(0x80000000).view(np.int32))]
        f.write(nodes.astype(np.int32).tobytes())
        pts = np.zeros((n, nv * 4), np.float32)
        pts[:, dp] = np.asarray(ids, np.int32).view(np.float32)
        f.write(pts.tobytes())


@pytest.mark.parametrize("case", ["magic", "truncated", "dup_ids", "range_ids", "bad_child"])
def test_load_refuses_bad_files(tmp_path, case):
    P = _lib()
    path = str(tmp_path / "t.bin")
    n, d, dp, nv, ns = 4, 3, 3, 1, 3
    if case == "magic":
        with open(path, "wb") as f:
            f.write(b"NOTATREE" + b"\0" * 200)
    elif case == "truncated":
        _write(path, n, d, dp, nv, ns, 1, [0, 1, 2, 3])
        with open(path, "r+b") as f:
            f.truncate(os.path.getsize(path) - 8)
    elif case == "dup_ids":
        _write(path, n, d, dp, nv, ns, 1, [0, 1, 1, 3])
    elif case == "range_ids":
        _write(path, n, d, dp, nv, ns, 1, [0, 1, 2, 9])
    else:
        nodes = np.zeros((1, ns * 4), np.int32)
        nodes[0, :4] = [5, 0, 0, 0]                       # inner node whose children lie outside
        _write(path, n, d, dp, nv, ns, 1, [0, 1, 2, 3], nodes)
    with pytest.raises(P.PandaError) as e:
        P.load_tree(path)
    assert e.value.status == 1


@pytest.mark.gpu
def test_save_load_round_trip(tmp_path):
    import torch
    P = _lib()
    P.load()
    pts = workloads.cosmology_points(150_000, seed=33, halos=25)
    t = P.build(torch.from_numpy(pts).cuda(), 32)
    path = str(tmp_path / "tree.bin")
    P.save(t, path)
    u = P.load_tree(path)
    a, b = t.info(), u.info()
    for key in ("n", "d", "bucket", "num_nodes", "num_leaves", "depth", "node_slots"):
        assert a[key] == b[key]
    q = torch.from_numpy(workloads.cosmology_points(20_000, seed=34, halos=25)).cuda()
    for fn in (lambda tr: P.knn(tr, q, 9), lambda tr: P.knn_self(tr, 9), lambda tr: P.knn(tr, q, 9, order="morton")):
        x, y = fn(t), fn(u)
        torch.cuda.synchronize()
        assert torch.equal(x[0], y[0]) and torch.equal(x[1].view(torch.int32), y[1].view(torch.int32))


@pytest.mark.gpu
def test_inner_right_start_is_only_a_hint(tmp_path):
    """The all-points query walks down to each job's leaf by the inner nodes'
    second header word (the right child's first packed position).  A table
    whose inner nodes hold other values there (zeros: always right; random
    words) still answers exactly: the walk's far children and its path cover
    the whole tree whichever leaf it reaches."""
    import torch
    P = _lib()
    P.load()
    pts = workloads.cosmology_points(60_000, seed=35, halos=12)
    t = P.build(torch.from_numpy(pts).cuda(), 32)
    want = P.knn_self(t, 7)
    torch.cuda.synchronize()
    path = str(tmp_path / "tree.bin")
    P.save(t, path)
    raw = bytearray(open(path, "rb").read())
    hdr = struct.unpack_from("<12q", raw, len(MAGIC))
    ns, slots = hdr[5], hdr[7]
    off = len(MAGIC) + 12 * 8 + 32 * 4
    nodes = np.frombuffer(bytes(raw[off:off + slots * ns * 16]), np.int32).reshape(slots, ns * 4).copy()
    inner = (nodes[:, 3].view(np.uint32) & 0x80000000) == 0
    assert inner.sum() > 1000
    rng = np.random.default_rng(36)
    for variant in ("zero", "random"):
        nodes[inner, 1] = 0 if variant == "zero" else rng.integers(-2**31, 2**31 - 1, inner.sum())
        raw[off:off + nodes.nbytes] = nodes.tobytes()
        p2 = str(tmp_path / f"tree_{variant}.bin")
        with open(p2, "wb") as f:
            f.write(raw)
        u = P.load_tree(p2)
        got = P.knn_self(u, 7)
        torch.cuda.synchronize()
        assert torch.equal(got[0], want[0]) and torch.equal(got[1].view(torch.int32), want[1].view(torch.int32)), variant
        u.free()
    t.free()

"""Host-side pieces of bench.py that need no GPU: the algorithmic byte counts
behind the build kernels' HBM roofline, the per-level point counts they use,
and that the JSON line's launch count is the one taken around the timed region."""
import ast
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_level_active_points():
    import bench
    # preorder tree: root 100 points, children 60 / 40, grandchildren under the 60
    exp = {"count": np.array([100, 60, 30, 30, 40]), "depth": np.array([0, 1, 2, 2, 1])}
    assert bench.level_active_points(exp, 35) == [100, 100]      # depth 2 holds no node > 35
    assert bench.level_active_points(exp, 10) == [100, 100, 60]
    assert bench.level_active_points(exp, 100) == []


def test_build_algorithmic_bytes():
    import bench
    info = {"point_floats": 4, "num_nodes": 10, "node_floats": 12}
    act = [1000, 1000, 600]
    b, _ = bench.build_algorithmic_bytes("level.partition", act, 1000, 3, info)
    assert b == 2600 * 2 * (4 * 3 + 4)
    b, _ = bench.build_algorithmic_bytes("level.hist", act, 1000, 3, info)
    assert b == 2600 * 4
    b, _ = bench.build_algorithmic_bytes("subtree", act, 1000, 3, info)
    assert b == 1000 * (4 * 3 + 4 + 4 * 4) + 10 * 12 * 4
    b, _ = bench.build_algorithmic_bytes("transpose", act, 1000, 3, info)
    assert b == 1000 * (8 * 3 + 4)


def test_gpu_launches_is_the_timed_region_count():
    """The JSON line's gpu_launches must be the library's launch counter read
    around the timed steps, and no later assignment may rebind that name."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    fn = next(f for f in tree.body if isinstance(f, ast.FunctionDef) and f.name == "run_ours")
    value = None
    for node in ast.walk(fn):
        if isinstance(node, ast.Dict):
            for k, v in zip(node.keys, node.values):
                if isinstance(k, ast.Constant) and k.value == "gpu_launches":
                    value = v
    assert isinstance(value, ast.Name), "gpu_launches should name the timed-region count"
    binds = []
    for node in ast.walk(fn):
        targets = []
        if isinstance(node, ast.Assign):
            targets = node.targets
        elif isinstance(node, (ast.AugAssign, ast.AnnAssign)):
            targets = [node.target]
        elif isinstance(node, (ast.For, ast.comprehension)):
            targets = [node.target]
        for t in targets:
            for n in ast.walk(t):
                if isinstance(n, ast.Name) and n.id == value.id:
                    binds.append(node)
    assert len(binds) == 1, f"{value.id} is bound {len(binds)} times in run_ours"
    src = ast.unparse(binds[0].value)
    assert "kernel_launches()" in src

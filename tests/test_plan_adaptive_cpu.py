"""The library's adaptive cluster tree and block tree (ph_plan_adaptive, host only) against the
oracle's (oracle.tree with leaf_size), on the batching workload's kind of point set: a mixture of
anisotropic Gaussians in 3-D (and a uniform 2-D set).  Sizes, leaf sizes, near and far counts,
near entries and the translation classes across levels must all agree."""
import numpy as np
import pytest

from oracle import tree
from paper_2511_03109_gb300 import inputs


@pytest.mark.parametrize("points,leaf,eta", [
    (lambda: inputs.gaussian_mixture_points(6000, 3, 32, 1003), 128, float(np.sqrt(3.0))),
    (lambda: inputs.gaussian_mixture_points(3000, 2, 8, 1004), 40, 1.0),
    (lambda: inputs.uniform_points(2000, 2, 1005), 30, float(np.sqrt(2.0))),
])
def test_adaptive_plan_matches_the_oracle(points, leaf, eta):
    from paper_2511_03109_gb300 import ph

    P = points()
    counts, perm = ph.plan(P, 0, eta, leaf_size=leaf)
    root = tree.build_cluster_tree(P, None, leaf_size=leaf)
    nodes = tree.all_nodes(root)
    leaves = [c for c in nodes if c.is_leaf()]
    near, far = tree.build_block_tree(root, eta)
    assert counts["nodes"] == len(nodes) and counts["leaves"] == len(leaves)
    assert counts["depth"] == max(c.level for c in nodes)
    assert all(c.n <= leaf or c.level >= 20 for c in leaves)
    assert counts["near"] == len(near) and counts["far"] == len(far)
    assert counts["near_entries"] == sum(s.n * t.n for s, t in near)
    # translation classes: both levels and the offset of the source box in units of the finer side
    classes = set()
    for s, t in far:
        unit = min(s.hi[0] - s.lo[0], t.hi[0] - t.lo[0])
        classes.add((s.level, t.level) + tuple(int(round(v)) for v in (t.lo - s.lo) / unit))
    assert counts["far_keys"] == len(classes)
    # the cluster order: the oracle's leaves in depth-first order, each in ascending index order
    np.testing.assert_array_equal(perm, np.concatenate([c.idx for c in leaves]))

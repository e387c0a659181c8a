"""Pins for the oracle's cluster tree and block cluster tree (§3.2, §3.4)."""
import os

import numpy as np
import pytest

from oracle import tree
from paper_2511_03109_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _coverage(root, n, eta):
    near, far = tree.build_block_tree(root, eta)
    cover = np.zeros((n, n), dtype=np.int32)
    for s, t in near + far:
        cover[np.ix_(s.idx, t.idx)] += 1
    return near, far, cover


@pytest.mark.parametrize("n,d,l_max,eta", [(300, 2, 3, 1.0), (257, 2, 2, np.sqrt(2.0)),
                                           (400, 3, 2, np.sqrt(3.0)), (64, 1, 4, 1.0)])
def test_partition_and_block_coverage(n, d, l_max, eta):
    P = inputs.uniform_points(n, d, 11 + n)
    root = tree.build_cluster_tree(P, l_max)
    lv = tree.leaves(root)
    seen = np.zeros(n, dtype=np.int32)
    for c in lv:
        seen[c.idx] += 1
        x = P[c.idx]
        assert np.all(x >= c.lo) and np.all(x <= c.hi)
        assert np.all(np.diff(c.idx) > 0)  # order inherited from I
        assert c.level == l_max
    assert np.all(seen == 1)
    near, far, cover = _coverage(root, n, eta)
    assert np.all(cover == 1)  # every (i, j) in exactly one block
    leafset = {id(c) for c in lv}
    for s, t in near:
        assert id(s) in leafset and id(t) in leafset  # D subset of L x L (§3.4)
    for s, t in far:
        assert s.level == t.level  # far pairs on one level (§3.4)
        assert max(tree.diam(s), tree.diam(t)) <= eta * tree.dist(s, t) * (1 + 1e-12)
    # sparsity constant bound C_sp <= 3^d 2^d for eta = sqrt(d) (§3.4)
    if abs(eta - np.sqrt(d)) < 1e-12:
        per = {}
        for s, t in near + far:
            per[id(s)] = per.get(id(s), 0) + 1
        assert max(per.values()) <= 3 ** d * 2 ** d


def test_split_plane_goes_low():
    P = np.array([[0.5, 0.25], [0.5000000001, 0.75], [0.0, 1.0], [1.0, 0.0]])
    root = tree.build_cluster_tree(P, 1)
    where = {}
    for c in root.children:
        for i in c.idx:
            where[int(i)] = tuple(c.halves)
    assert where[0] == (0, 0) and where[1] == (1, 1) and where[2] == (0, 1) and where[3] == (1, 0)


def test_admissibility_ties_and_touching():
    a = tree.Cluster([], [0, 0, 0], [0.25, 0.25, 0.25], 2)
    b = tree.Cluster([], [0.5, 0, 0], [0.75, 0.25, 0.25], 2)  # one-box gap along x
    c = tree.Cluster([], [0.25, 0.25, 0], [0.5, 0.5, 0.25], 2)  # touches a at an edge
    assert tree.dist(a, c) == 0.0 and not tree.admissible(a, c, np.sqrt(3))
    assert tree.admissible(a, b, np.sqrt(3.0))  # diam = sqrt(3) h = eta * dist: tie is admissible
    assert not tree.admissible(a, b, 1.5)


def _golden_ratios():
    rows = []
    with open(os.path.join(GOLDEN, "nf_ratio.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, l, r, tol = line.split()
                rows.append((int(n), int(l), float(r), float(tol)))
    return rows


@pytest.mark.parametrize("n,l_max,ratio,tol", [r for r in _golden_ratios() if r[0] <= 100000])
def test_near_field_ratio_matches_paper(n, l_max, ratio, tol):
    P = inputs.uniform_points(n, 3, 4242)
    root = tree.build_cluster_tree(P, l_max)
    near, far = tree.build_block_tree(root, np.sqrt(3.0))
    side = 2 ** l_max
    # with eta = sqrt(3) the near pairs are exactly the neighbouring boxes: (3 side - 2)^3
    assert len(near) == (3 * side - 2) ** 3
    got = sum(s.n * t.n for s, t in near) / float(n) ** 2
    assert abs(got - ratio) / ratio < tol


@pytest.mark.parametrize("d,leaf", [(2, 16), (3, 20)])
def test_adaptive_tree_leaf_rule_coverage_and_empty_children(d, leaf):
    """Adaptive mode (leaf_size): a node is split while it holds more than leaf_size points
    and is above max_depth; empty children are dropped; every point lies in exactly one leaf,
    inside its box; the block tree still covers every (i, j) exactly once."""
    rng = np.random.default_rng(17 + d)
    # two tight clusters plus a uniform background: uneven depths and empty children
    P = np.clip(np.concatenate([0.3 + 0.01 * rng.standard_normal((150, d)),
                                0.8 + 0.002 * rng.standard_normal((90, d)),
                                rng.random((60, d))]), 0.0, 1.0)
    n = P.shape[0]
    root = tree.build_cluster_tree(P, 0, leaf_size=leaf, max_depth=12)
    lv = tree.leaves(root)
    seen = np.zeros(n, dtype=np.int32)
    depths = set()
    for c in lv:
        seen[c.idx] += 1
        assert c.n >= 1  # empty children are dropped
        assert c.n <= leaf or c.level == 12
        assert np.all(P[c.idx] >= c.lo) and np.all(P[c.idx] <= c.hi)
        depths.add(c.level)
    assert np.all(seen == 1)
    assert len(depths) > 1  # the tree is not uniform
    for c in tree.all_nodes(root):
        if c.children:
            assert c.n > leaf
            assert sum(ch.n for ch in c.children) == c.n
            assert len(c.children) <= 2 ** d
            for ch in c.children:
                np.testing.assert_allclose(ch.hi - ch.lo, 0.5 * (c.hi - c.lo))
    # points of one cell of the finest split that hold only duplicates stop at max_depth
    dup = np.concatenate([np.full((leaf + 5, d), 0.123), rng.random((10, d))])
    r2 = tree.build_cluster_tree(dup, 0, leaf_size=leaf, max_depth=6)
    assert max(c.level for c in tree.leaves(r2)) == 6
    near, far, cover = _coverage(root, n, np.sqrt(d))
    assert np.all(cover == 1)
    for s, t in near:
        assert s.is_leaf() or t.is_leaf()  # recursion stops when either side is a leaf


@pytest.mark.parametrize("n,l_max,ratio,tol", _golden_ratios())
def test_library_planner_near_field_ratio_matches_paper(n, l_max, ratio, tol):
    """The library's host planner (ph_plan) gives the paper's NF Ratio column too, up to the
    sampling noise of a fresh uniform draw, including n = 8^6."""
    from paper_2511_03109_gb300 import ph

    P = inputs.uniform_points(n, 3, 4242)
    counts, _ = ph.plan(P, l_max, np.sqrt(3.0))
    side = 2 ** l_max
    assert counts["near"] == (3 * side - 2) ** 3
    assert abs(counts["near_entries"] / float(n) ** 2 - ratio) / ratio < tol

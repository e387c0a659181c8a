"""Cluster tree, admissibility and block cluster tree (§3.2, §3.4, App. A.1, A.2).

Test infrastructure only (see ``oracle/__init__.py``).

Readings taken where the paper is garbled or silent:

* Alg. ConstructClusterTree stops on "level > l_max" and recurses with
  "l_max + 1", which contradicts "all leaves are at level l_max" (§3.2).  Here a
  node is split while its level is below l_max, and l_max is passed unchanged.
* The root box is B = [0, 1]^d (the paper's domain, §6), not the bounding box.
* Splits are at the midpoint with the low half closed and the high half
  half-open: [a, mid] and (mid, b] (App. A.1), so a point on a split plane goes
  to the low child.
* Children are enumerated in little-endian order of their per-dimension halves
  (dimension 1 fastest), matching the flattening of §2.1.
* Empty children are dropped (they contribute no rows or columns).
* Admissibility (§3.4): max(diam B_s, diam B_t) <= eta * dist(B_s, B_t) with
  diam and dist of App. A.2.  Boxes are closed, so touching boxes have distance
  zero.  Equality counts as admissible; the comparison carries a relative
  slack of 1e-12 so that exact ties (e.g. eta = sqrt(d) at a one-box gap) do not
  depend on rounding.

Pins (tests/test_oracle_tree.py): every point in exactly one leaf and inside
its box; every (i, j) covered by exactly one near or far block (brute force);
near blocks are leaf x leaf and far blocks pair clusters of equal level (§3.4);
for the uniform d = 3, eta = sqrt(3) tree the near pairs are exactly the
neighbouring boxes (10^3 at l_max = 2, 22^3 at l_max = 3) and the near-field
ratio matches the paper's NF Ratio column within sampling noise.
"""
from __future__ import annotations

import numpy as np

ADMISSIBILITY_SLACK = 1e-12


class Cluster:
    """A node sigma of the cluster tree: index set I_sigma (ascending), box B_sigma, level."""

    def __init__(self, idx, lo, hi, level, parent=None, halves=None):
        self.idx = np.asarray(idx, dtype=np.int64)
        self.lo = np.asarray(lo, float)
        self.hi = np.asarray(hi, float)
        self.level = int(level)
        self.parent = parent
        self.halves = halves  # per-dimension 0 (low) / 1 (high) position inside the parent box
        self.children = []
        self.id = -1

    @property
    def n(self) -> int:
        return int(self.idx.size)

    def is_leaf(self) -> bool:
        return not self.children


def build_cluster_tree(points: np.ndarray, l_max: int, lo=None, hi=None, leaf_size=None,
                       max_depth: int = 20) -> Cluster:
    """Cluster tree T_I of §3.2 by recursive midpoint bisection (Alg. ConstructClusterTree).

    Uniform mode (leaf_size is None): every non-empty node above level l_max is split.
    Adaptive mode: a node is split while it holds more than leaf_size points and
    its level is below max_depth.
    """
    P = np.asarray(points, float)
    n, d = P.shape
    lo = np.zeros(d) if lo is None else np.asarray(lo, float)
    hi = np.ones(d) if hi is None else np.asarray(hi, float)
    if np.any(P < lo) or np.any(P > hi):
        raise ValueError("points must lie in the root box")
    root = Cluster(np.arange(n), lo, hi, 0)

    def split(node: Cluster):
        if leaf_size is None:
            if node.level >= l_max:
                return
        elif node.n <= leaf_size or node.level >= max_depth:
            return
        mid = 0.5 * (node.lo + node.hi)
        x = P[node.idx]
        upper = x > mid  # (mid, b] is the high half
        for t in range(2 ** d):
            halves = [(t >> k) & 1 for k in range(d)]
            mask = np.ones(node.n, dtype=bool)
            clo, chi = node.lo.copy(), node.hi.copy()
            for k in range(d):
                if halves[k]:
                    mask &= upper[:, k]
                    clo[k] = mid[k]
                else:
                    mask &= ~upper[:, k]
                    chi[k] = mid[k]
            if not mask.any():
                continue
            child = Cluster(node.idx[mask], clo, chi, node.level + 1, parent=node, halves=halves)
            node.children.append(child)
        for c in node.children:
            split(c)

    split(root)
    number_nodes(root)
    return root


def number_nodes(root: Cluster) -> list:
    """Give every node an id in depth-first pre-order and return the node list."""
    nodes = []

    def walk(c):
        c.id = len(nodes)
        nodes.append(c)
        for ch in c.children:
            walk(ch)

    walk(root)
    return nodes


def all_nodes(root: Cluster) -> list:
    out = []

    def walk(c):
        out.append(c)
        for ch in c.children:
            walk(ch)

    walk(root)
    return out


def leaves(root: Cluster) -> list:
    return [c for c in all_nodes(root) if c.is_leaf()]


def diam(c: Cluster) -> float:
    """diam(B) = (sum_i (b_i - a_i)^2)^(1/2) (App. A.2)."""
    return float(np.sqrt(np.sum((c.hi - c.lo) ** 2)))


def dist(s: Cluster, t: Cluster) -> float:
    """dist(B1, B2) = (sum_i max(0, a_i - d_i)^2 + max(0, c_i - b_i)^2)^(1/2) (App. A.2)."""
    g1 = np.maximum(0.0, s.lo - t.hi)
    g2 = np.maximum(0.0, t.lo - s.hi)
    return float(np.sqrt(np.sum(g1 * g1 + g2 * g2)))


def admissible(s: Cluster, t: Cluster, eta: float) -> bool:
    """Strong admissibility of §3.4 (equality admissible, see module docstring)."""
    return max(diam(s), diam(t)) <= eta * dist(s, t) * (1.0 + ADMISSIBILITY_SLACK)


def build_block_tree(root: Cluster, eta: float):
    """Leaves of the block cluster tree (Alg. ConstructBlockClusterTree, §3.4).

    Returns (near, far): lists of (sigma, tau) pairs, far = admissible leaves
    (the set A), near = inadmissible leaves (the set D), in depth-first order.
    """
    near, far = [], []

    def recurse(s: Cluster, t: Cluster):
        adm = admissible(s, t, eta)
        if not adm and s.children and t.children:
            for sc in s.children:
                for tc in t.children:
                    recurse(sc, tc)
        elif adm:
            far.append((s, t))
        else:
            near.append((s, t))

    recurse(root, root)
    return near, far

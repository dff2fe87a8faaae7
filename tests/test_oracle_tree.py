"""Pins for the oracle's root cube, Morton keys, octree and U/V/W/X lists.

Lists are checked against a brute-force classification of every box pair by
the definitions (paper §2.2: the interaction list is the children of the
parent's neighbours that are not neighbours; adaptive U/W/X lists of the
cited kernel-independent FMM paper), and by the partition invariant: every
(target leaf, source point) pair is reached by exactly one list.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1602_02244_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_morton_golden_hand_derived():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_keys.txt")) if l.strip() and not l.startswith("#")]
    xyz = np.array([[float(v) for v in r[:3]] for r in rows])
    want = np.array([int(r[3]) for r in rows], dtype=np.uint64)
    lo, D = oracle.root_cube(xyz)
    assert tuple(lo) == (0.0, 0.0, 0.0) and D == 1.0
    np.testing.assert_array_equal(oracle.morton_keys(xyz, lo, D), want)


@pytest.mark.parametrize("ext,D", [(0.999, 1.0), (1.0, 2.0), (0.5, 1.0), (0.49, 0.5), (19.7, 32.0), (0.0, 1.0)])
def test_root_cube_smallest_power_of_two_above_extent(ext, D):
    xyz = np.array([[-3.0, 1.0, 2.0], [-3.0 + ext, 1.0, 2.0 + ext / 3]])
    lo, d = oracle.root_cube(xyz)
    assert tuple(lo) == (-3.0, 1.0, 2.0)
    assert d == D


def test_root_cube_rejects_nonfinite():
    with pytest.raises(ValueError):
        oracle.root_cube(np.array([[0.0, np.nan, 1.0]]))


def test_keys_place_points_inside_their_boxes():
    """For every point and level l, the key prefix key >> 3(21-l) decodes to
    the anchor of a box of side D/2^l that contains the point (catches a
    swapped axis or a wrong bit order)."""
    xyz = workloads.plummer(2000, seed=4)
    lo, D = oracle.root_cube(xyz)
    keys = oracle.morton_keys(xyz, lo, D).astype(object)
    for l in (1, 3, 7, 12, 21):
        a = D / 2 ** l
        for i in range(0, 2000, 37):
            pre = int(keys[i]) >> (3 * (21 - l))
            anc = [0, 0, 0]
            for b in range(l):
                for ax in range(3):
                    anc[ax] |= ((pre >> (3 * b + ax)) & 1) << b
            for ax in range(3):
                lo_b = lo[ax] + anc[ax] * a
                assert lo_b - 1e-12 * D <= xyz[i, ax] <= lo_b + a + 1e-12 * D


# ------------------------------------------------------------------ brute force
class Boxes:
    def __init__(self, t):
        self.t = t
        self.nb = t.nboxes
        self.level = t.box_level
        self.anc = [t.anchor(b) for b in range(self.nb)]
        self.leaf = t.box_nchild == 0

    def adjacent(self, A, B):
        la, lb = int(self.level[A]), int(self.level[B])
        for ax in range(3):
            alo, ahi = self.anc[A][ax] << (21 - la), (self.anc[A][ax] + 1) << (21 - la)
            blo, bhi = self.anc[B][ax] << (21 - lb), (self.anc[B][ax] + 1) << (21 - lb)
            if alo > bhi or blo > ahi:
                return False
        return True

    def ancestor_at(self, A, l):
        while self.level[A] > l:
            A = int(self.t.box_parent[A])
        return A


def brute_lists(t):
    bx = Boxes(t)
    nb = bx.nb
    U, V, W, X = ([[] for _ in range(nb)] for _ in range(4))
    for B in range(nb):
        lB = int(bx.level[B])
        for A in range(nb):
            lA = int(bx.level[A])
            adj = bx.adjacent(A, B)
            if lB >= 2 and lA == lB and not adj:
                if bx.adjacent(int(t.box_parent[A]), int(t.box_parent[B])):
                    V[B].append(A)
            if bx.leaf[B]:
                if bx.leaf[A] and adj:
                    U[B].append(A)
                if lA > lB and not adj and bx.adjacent(int(t.box_parent[A]), B):
                    C = bx.ancestor_at(A, lB)
                    if C != B and bx.adjacent(C, B):
                        W[B].append(A)
    for B in range(nb):
        for A in W[B]:
            X[A].append(B)
    return U, V, W, [sorted(x) for x in X]


def direct_wx_lists(t, lists, max_points):
    """The lists after moving each W pair of two leaves whose W leaf holds at
    most max_points points to the near field, in both directions."""
    U, V, W, X = ([list(r) for r in rows] for rows in lists)
    leaf = t.box_nchild == 0
    for B in range(t.nboxes):
        for A in list(W[B]):
            if leaf[A] and t.box_count[A] <= max_points:
                W[B].remove(A)
                X[A].remove(B)
                U[B].append(A)
                U[A].append(B)
    return [sorted(u) for u in U], V, W, X


def _inputs(kind, n, seed):
    if kind == "uniform":
        return workloads.uniform_cube(n, seed)
    if kind == "plummer":
        return workloads.plummer(n, seed)
    return workloads.sphere_surface(n, seed)


@pytest.mark.parametrize("kind,n,S", [("uniform", 600, 8), ("plummer", 500, 6), ("sphere", 400, 5),
                                       ("uniform", 64, 64), ("plummer", 300, 1)])
def test_lists_equal_brute_force(kind, n, S):
    xyz = _inputs(kind, n, seed=11)
    t = oracle.Tree(xyz, S)
    U, V, W, X = brute_lists(t)
    for name, ref in (("u", U), ("v", V), ("w", W), ("x", X)):
        for b in range(t.nboxes):
            assert list(t.lst(name, b)) == ref[b], (name, b)


@pytest.mark.parametrize("kind,n,S", [("plummer", 500, 6), ("sphere", 400, 5), ("plummer", 300, 1)])
def test_direct_wx_lists_equal_brute_force(kind, n, S):
    xyz = _inputs(kind, n, seed=11)
    t0 = oracle.Tree(xyz, S)
    for d in (1, 4, 81):
        t = oracle.Tree(xyz, S, direct_wx=d)
        ref = direct_wx_lists(t0, brute_lists(t0), d)
        for name, rows in zip("uvwx", ref):
            for b in range(t.nboxes):
                assert list(t.lst(name, b)) == rows[b], (d, name, b)


@pytest.mark.parametrize("kind,n,S,direct", [("uniform", 2000, 12, 0), ("plummer", 2000, 10, 0),
                                             ("sphere", 1500, 7, 0), ("plummer", 2000, 10, 81),
                                             ("sphere", 1500, 7, 10 ** 6), ("plummer", 3000, 4, 3)])
def test_lists_partition_every_pair_exactly_once(kind, n, S, direct):
    """Each (leaf B target, source point j) pair is reached exactly once by
    P2P over U(B), M2P over W(B), or M2L over V(C) / P2L over X(C) for C = B
    or an ancestor of B -- also after small W/X leaf pairs moved to U, whose
    rows stay symmetric (A in U(B) iff B in U(A))."""
    xyz = _inputs(kind, n, seed=5)
    t = oracle.Tree(xyz, S, direct_wx=direct)
    for B in np.nonzero(t.box_nchild == 0)[0]:
        for A in t.lst("u", B):
            assert B in t.lst("u", A)
    first, cnt = t.box_first, t.box_count
    for B in np.nonzero(t.box_nchild == 0)[0]:
        hit = np.zeros(n, np.int32)
        for A in list(t.lst("u", B)) + list(t.lst("w", B)):
            hit[first[A]:first[A] + cnt[A]] += 1
        C = int(B)
        while C >= 0:
            for A in list(t.lst("v", C)) + list(t.lst("x", C)):
                hit[first[A]:first[A] + cnt[A]] += 1
            C = int(t.box_parent[C])
        assert np.all(hit == 1), (B, np.unique(hit))


def test_tree_structure_invariants():
    xyz = workloads.plummer(3000, seed=9)
    S = 16
    t = oracle.Tree(xyz, S)
    lo, D = oracle.root_cube(xyz)
    # stable sort by key
    keys = oracle.morton_keys(xyz, lo, D)
    order = np.lexsort((np.arange(len(keys)), keys))
    np.testing.assert_array_equal(t.perm, order)
    np.testing.assert_array_equal(t.keys, keys[order])
    # leaves respect the leaf size; children are non-empty and partition parents
    leaf = t.box_nchild == 0
    assert np.all(t.box_count[leaf] <= S)
    assert np.all(t.box_count >= 1)
    for b in np.nonzero(~leaf)[0]:
        ch = range(t.box_child[b], t.box_child[b] + t.box_nchild[b])
        assert sum(t.box_count[c] for c in ch) == t.box_count[b]
        assert all(t.box_parent[c] == b for c in ch)
        assert t.box_count[b] > S
    # index order = (level, key)
    lk = list(zip(t.box_level.tolist(), t.box_key.tolist()))
    assert lk == sorted(lk)
    # |V| <= 189 and V offsets inside the 316 well-separated offsets
    for b in range(t.nboxes):
        v = t.lst("v", b)
        assert len(v) <= 189
        ab = np.array(t.anchor(b))
        for a in v:
            d = np.array(t.anchor(a)) - ab
            assert np.abs(d).max() in (2, 3)


def test_uniform_tree_has_no_w_x_and_27_neighbours():
    """A lattice with 8 points per level-3 box gives a uniform tree."""
    g = (np.arange(16) + 0.5) / 16.0
    xyz = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    t = oracle.Tree(xyz, 8)
    assert set(t.box_level[t.box_nchild == 0].tolist()) == {3}
    assert len(t.w_idx) == 0 and len(t.x_idx) == 0
    u = np.diff(t.u_off)[t.box_nchild == 0]
    assert u.max() == 27 and u.min() == 8
    v = np.diff(t.v_off)[t.level_offset[3]:t.level_offset[4]]
    assert v.max() == 189


def test_leaf_may_exceed_leaf_size_only_at_max_depth():
    xyz = np.zeros((40, 3))
    xyz[:, 0] = np.linspace(0, 1e-9, 40)
    xyz = np.vstack([xyz, [[1.0, 1.0, 1.0]]])
    t = oracle.Tree(xyz, 4, max_depth=21)
    big = (t.box_nchild == 0) & (t.box_count > 4)
    assert np.all(t.box_level[big] == 21)
    t2 = oracle.Tree(xyz, 4, max_depth=5)
    assert t2.nlevels == 6
    assert t2.box_count[(t2.box_nchild == 0)].max() > 4


def test_empty_and_single_point():
    t0 = oracle.Tree(np.zeros((0, 3)), 8)
    assert t0.nboxes == 0
    t1 = oracle.Tree(np.array([[0.3, 0.2, 0.1]]), 8)
    assert t1.nboxes == 1 and list(t1.lst("u", 0)) == [0]
    phi, g = t1.eval(4, np.array([2.0]))
    assert phi[0] == 0.0 and np.all(g == 0.0)

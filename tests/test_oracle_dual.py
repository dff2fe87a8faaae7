"""Pins for the oracle's dual-tree walk and its FMM (§2.1: the dual tree walk
with a multipole acceptance criterion, after Dehnen, as the alternative to
fixed interaction lists).

The walk is pinned by what its definition fixes independently of how it is
coded: the cover of all (target point, source point) pairs exactly once, the
acceptance criterion on both sides of every decision, the symmetry of the
pair sets, and the cell radii recomputed from the points.  The FMM on its
lists is pinned by the direct sum it must reproduce when nothing is accepted
(theta = 0), by geometric convergence in the order p, and by the symmetry of
the truncated operator (column probe).
"""
import numpy as np
import pytest

import oracle
from paper_1602_02244_gb300 import workloads


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def centres(t):
    """Box centres lo + (anchor + 1/2) a, elementwise IEEE like the definition."""
    anc = np.array([t.anchor(b) for b in range(t.nboxes)], dtype=np.float64)
    a = t.D * np.ldexp(1.0, -t.box_level.astype(np.int64))
    return t.lo[None, :] + (anc + 0.5) * a[:, None], anc, a


def accept(anc, a, r, theta, T, S):
    d = (anc[T] + 0.5) * a[T] - (anc[S] + 0.5) * a[S]  # exact: dyadic centres
    dist = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    return r[T] + r[S] < theta * dist


def pairs(d, name, nb):
    off = getattr(d, name + "_off")
    idx = getattr(d, name + "_idx")
    rows = np.repeat(np.arange(nb), np.diff(off))
    return set(zip(rows.tolist(), idx.tolist()))


@pytest.fixture(scope="module", params=["plummer", "uniform"])
def small(request):
    if request.param == "plummer":
        xyz, _ = workloads.plummer_problem(700, seed=11)
    else:
        xyz = workloads.rng(12).uniform(0, 1, (700, 3))
    return oracle.Tree(xyz, 6)


@pytest.mark.parametrize("theta", [0.35, 0.6, 0.9])
def test_every_point_pair_covered_exactly_once(small, theta):
    t = small
    d = oracle.Dual(t, theta)
    n = t.n
    cover = np.zeros((n, n), np.int32)  # sorted target index x sorted source index
    f, c = t.box_first, t.box_count
    for name in ("m2l", "p2p"):
        for T, S in pairs(d, name, t.nboxes):
            cover[f[T]:f[T] + c[T], f[S]:f[S] + c[S]] += 1
    assert cover.min() == 1 and cover.max() == 1


@pytest.mark.parametrize("theta", [0.35, 0.6, 0.9])
def test_acceptance_criterion_and_split_rule(small, theta):
    t = small
    d = oracle.Dual(t, theta)
    _, anc, a = centres(t)
    r = d.radius
    leaf = t.box_nchild == 0
    m2l = pairs(d, "m2l", t.nboxes)
    p2p = pairs(d, "p2p", t.nboxes)
    assert m2l and p2p
    for T, S in m2l:
        assert T != S and accept(anc, a, r, theta, T, S)
        # the cells never overlap: neither is an ancestor of the other
        for X, Y in ((T, S), (S, T)):
            while X >= 0:
                assert X != Y
                X = t.box_parent[X]
    for T, S in p2p:
        assert leaf[T] and leaf[S]
        assert T == S or not accept(anc, a, r, theta, T, S)
    # symmetric pair sets: the truncated operator is symmetric
    assert m2l == {(S, T) for T, S in m2l}
    assert p2p == {(S, T) for T, S in p2p}
    # every leaf meets itself in P2P
    assert all((b, b) in p2p for b in np.flatnonzero(leaf))


def test_radius_is_farthest_point_from_centre(small):
    t = small
    d = oracle.Dual(t, 0.5)
    c, _, _ = centres(t)
    for b in range(t.nboxes):
        x = t.xyz[t.perm[t.box_first[b]:t.box_first[b] + t.box_count[b]]]
        dx = x - c[b]
        s = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]
        assert d.radius[b] == np.sqrt(s.max())


def test_radius_of_a_single_point_box_is_its_offset():
    xyz = np.array([[0.1, 0.2, 0.3], [0.9, 0.8, 0.7]])
    t = oracle.Tree(xyz, 1)
    d = oracle.Dual(t, 0.5)
    c, _, _ = centres(t)
    for b in range(t.nboxes):
        if t.box_count[b] == 1:
            i = t.perm[t.box_first[b]]
            assert d.radius[b] == np.sqrt(((xyz[i] - c[b]) ** 2).sum())


def test_theta_zero_is_the_direct_sum():
    """Nothing is accepted: every point pair goes through P2P of leaves."""
    xyz, _ = workloads.plummer_problem(1500, seed=2)
    q = workloads.rng(3).uniform(-1, 1, 1500)
    t = oracle.Tree(xyz, 16)
    d = oracle.Dual(t, 0.0)
    assert len(d.m2l_idx) == 0
    phi, g = d.eval(6, q)
    phi_d, g_d = oracle.direct(xyz, q)
    assert rel(phi, phi_d) < 1e-13 and rel(g, g_d) < 1e-13


def test_converges_geometrically_in_p_with_cross_level_m2l():
    """Pairs of cells of different sizes carry a large part of the far field;
    the error falls by a fixed factor per order and theta orders it."""
    xyz, _ = workloads.plummer_problem(3000, seed=1)
    q = workloads.rng(5).uniform(-1, 1, 3000)
    t = oracle.Tree(xyz, 16)
    phi_d, g_d = oracle.direct(xyz, q)
    errs = {}
    for theta in (0.3, 0.5):
        d = oracle.Dual(t, theta)
        lv = t.box_level
        rows = np.repeat(np.arange(t.nboxes), np.diff(d.m2l_off))
        assert np.count_nonzero(lv[rows] != lv[d.m2l_idx]) > len(d.m2l_idx) // 5
        e = []
        for p in (2, 4, 6, 8, 10):
            phi, g = d.eval(p, q)
            e.append((rel(phi, phi_d), rel(g, g_d)))
        for (a, ga), (b, gb) in zip(e, e[1:]):
            assert b < a / 3 and gb < ga / 3
        errs[theta] = e
    assert errs[0.3][-1][0] < 1e-8 and errs[0.5][-1][0] < 5e-6
    assert all(x[0] < y[0] for x, y in zip(errs[0.3], errs[0.5]))


def test_truncated_operator_is_symmetric():
    xyz, _ = workloads.plummer_problem(150, seed=3)
    t = oracle.Tree(xyz, 4)
    d = oracle.Dual(t, 0.6)
    assert len(d.m2l_idx) > 1000
    A = np.zeros((150, 150))
    for j in range(150):
        e = np.zeros(150)
        e[j] = 1.0
        A[:, j] = d.eval(4, e, grad=False)
    assert np.linalg.norm(A - A.T) / np.linalg.norm(A) < 1e-13

"""Pins for the oracle's direct sum, solid harmonics and single translations.

Each check compares the oracle with something other than itself: closed forms,
scipy's associated Legendre functions, invariances of the Laplace kernel, the
Greengard-Rokhlin truncation bound, exactness of re-expansions, or finite
differences of the oracle's own potential field.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def idx(n, m):
    return n * n + n + m


# ---------------------------------------------------------------- harmonics
@pytest.mark.parametrize("x", [(0.3, -0.2, 0.5), (-1.1, 0.4, -0.3), (0.0, 0.0, 2.0), (0.7, 0.7, 0.0)])
def test_harmonics_match_legendre(x):
    """R_n^m = r^n P_n^m(cos t) e^{imp}/(n+m)!, I_n^m = (n-m)! P_n^m e^{imp}/r^{n+1}
    with scipy's Condon-Shortley P_n^m, and the (-1)^m conj symmetry for m < 0."""
    from scipy.special import lpmv
    p = 10
    x = np.array(x)
    r = np.linalg.norm(x)
    ct = x[2] / r
    ph = math.atan2(x[1], x[0])
    R = oracle.regular(p, x)
    I = oracle.irregular(p, x)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            P = lpmv(am, n, ct)
            if m >= 0:
                rr = r ** n * P * np.exp(1j * m * ph) / math.factorial(n + m)
                ii = math.factorial(n - m) * P * np.exp(1j * m * ph) / r ** (n + 1)
            else:
                rr = (-1) ** am * np.conj(r ** n * P * np.exp(1j * am * ph) / math.factorial(n + am))
                ii = (-1) ** am * np.conj(math.factorial(n - am) * P * np.exp(1j * am * ph) / r ** (n + 1))
            assert abs(R[idx(n, m)] - rr) <= 1e-12 * max(1.0, abs(rr))
            assert abs(I[idx(n, m)] - ii) <= 1e-12 * max(1.0, abs(ii))


def test_addition_theorem_reproduces_coulomb():
    """1/|x-y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x) for |y| < |x| (series converges
    geometrically in |y|/|x|)."""
    x = np.array([1.0, 0.7, -0.4])
    y = np.array([0.1, -0.2, 0.15])
    p = 40
    s = np.sum(np.conj(oracle.regular(p, y)) * oracle.irregular(p, x))
    assert abs(s.imag) < 1e-14
    assert abs(s.real - 1 / np.linalg.norm(x - y)) < 1e-14


def test_regular_addition_theorem():
    """R_n^m(a+b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b) (finite, exact)."""
    p = 8
    rng = np.random.default_rng(5)
    a, b = rng.normal(size=3) * 0.4, rng.normal(size=3) * 0.4
    Ra, Rb, Rab = oracle.regular(p, a), oracle.regular(p, b), oracle.regular(p, a + b)

    def g(R, n, m):
        return R[idx(n, m)] if 0 <= n and abs(m) <= n else 0.0
    for n in range(p + 1):
        for m in range(-n, n + 1):
            s = sum(g(Ra, k, l) * g(Rb, n - k, m - l) for k in range(n + 1) for l in range(-k, k + 1))
            assert abs(s - Rab[idx(n, m)]) < 1e-13


# --------------------------------------------------------------- direct sum
def test_direct_two_particles_closed_form():
    """phi = q/r and grad phi = -q (x_t - x_s)/r^3 for one source."""
    src = np.array([[0.1, 0.2, -0.3], [1.1, -0.8, 0.9]])
    q = np.array([0.7, -1.3])
    phi, g = oracle.direct(src, q)
    d = src[0] - src[1]
    r = np.linalg.norm(d)
    assert phi[0] == pytest.approx(q[1] / r, rel=1e-15)
    assert phi[1] == pytest.approx(q[0] / r, rel=1e-15)
    np.testing.assert_allclose(g[0], -q[1] * d / r ** 3, rtol=1e-14)
    np.testing.assert_allclose(g[1], q[0] * d / r ** 3, rtol=1e-14)


def test_direct_octahedron_centre():
    """Six unit charges at distance 2 on the axes: phi(0) = 3, grad(0) = 0."""
    src = 2.0 * np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    phi, g = oracle.direct(src, np.ones(6), np.zeros((1, 3)))
    assert phi[0] == pytest.approx(3.0, rel=1e-15)
    assert np.abs(g).max() < 1e-15


def test_direct_coincident_points_contribute_nothing():
    src = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    phi, g = oracle.direct(src, np.array([1.0, 2.0, 4.0]))
    assert phi[0] == pytest.approx(4.0)
    assert phi[1] == pytest.approx(4.0)
    assert phi[2] == pytest.approx(3.0)


def test_direct_symmetry_invariances_and_fd():
    """w.(K q) = q.(K w) (K symmetric); translation, rotation and scaling
    covariance; gradient = central FD of the potential."""
    rng = np.random.default_rng(1)
    x = rng.random((300, 3))
    q = rng.uniform(-1, 1, 300)
    w = rng.normal(size=300)
    pq, gq = oracle.direct(x, q)
    pw, _ = oracle.direct(x, w)
    assert abs(w @ pq - q @ pw) <= 1e-13 * abs(w @ pq)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    p2, g2 = oracle.direct(x @ Q.T * 2.5 + np.array([3.0, -1.0, 7.0]), q)
    np.testing.assert_allclose(p2, pq / 2.5, rtol=1e-12)
    np.testing.assert_allclose(g2, gq @ Q.T / 2.5 ** 2, rtol=1e-9, atol=1e-12 * np.abs(gq).max())
    h = 1e-5
    for i in (0, 17, 123):
        for a in range(3):
            xp, xm = x[i].copy(), x[i].copy()
            xp[a] += h
            xm[a] -= h
            src = np.delete(x, i, axis=0)
            qs = np.delete(q, i)
            fp = oracle.direct(src, qs, xp[None])[0][0]
            fm = oracle.direct(src, qs, xm[None])[0][0]
            assert (fp - fm) / (2 * h) == pytest.approx(gq[i, a], rel=1e-6, abs=1e-8)


# ---------------------------------------------------------- translations
def _cluster(rng, c, a, n):
    return c + a * (rng.random((n, 3)) - 0.5)


@pytest.mark.parametrize("p", [2, 4, 8, 12])
def test_p2m_m2p_within_greengard_rokhlin_bound(p):
    """|phi_direct - phi_M2P| <= sum|q| / (r - rho) * (rho/r)^(p+1)."""
    rng = np.random.default_rng(p)
    c = np.array([0.2, -0.1, 0.3])
    src = _cluster(rng, c, 1.0, 40)
    q = rng.uniform(-1, 1, 40)
    rho = np.linalg.norm(src - c, axis=1).max()
    tgt = c + rng.normal(size=(50, 3)) * 3
    tgt = tgt[np.linalg.norm(tgt - c, axis=1) > 2.0 * rho]
    M = oracle.p2m(p, c, src, q)
    phi, g = oracle.m2p(p, c, M, tgt)
    pd, gd = oracle.direct(src, q, tgt)
    r = np.linalg.norm(tgt - c, axis=1)
    bound = np.abs(q).sum() / (r - rho) * (rho / r) ** (p + 1)
    assert np.all(np.abs(phi - pd) <= bound * (1 + 1e-9) + 1e-15)


@pytest.mark.parametrize("p", [2, 4, 8, 12])
def test_p2l_l2p_within_local_expansion_bound(p):
    """Sources at distance >= rho from c, targets at r < rho:
    |phi_direct - phi_L2P(P2L)| <= sum|q| / (rho - r) * (r/rho)^(p+1)
    (the local-expansion error bound of Greengard and Rokhlin)."""
    rng = np.random.default_rng(20 + p)
    c = np.array([-0.3, 0.2, 0.1])
    d = rng.normal(size=(40, 3))
    src = c + d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(2.0, 4.0, (40, 1))
    q = rng.uniform(-1, 1, 40)
    rho = np.linalg.norm(src - c, axis=1).min()
    tgt = _cluster(rng, c, 1.6, 60)
    r = np.linalg.norm(tgt - c, axis=1)
    tgt, r = tgt[r < 0.9 * rho], r[r < 0.9 * rho]
    L = oracle.p2l(p, c, src, q)
    phi, _ = oracle.l2p(p, c, L, tgt)
    pd, _ = oracle.direct(src, q, tgt)
    bound = np.abs(q).sum() / (rho - r) * (r / rho) ** (p + 1)
    assert len(tgt) > 20
    assert np.all(np.abs(phi - pd) <= bound * (1 + 1e-9) + 1e-15)


@pytest.mark.parametrize("p", [0, 1, 3, 8, 15])
def test_single_charge_expansions_are_the_truncated_legendre_series(p):
    """One unit charge, expansions of degree p about c.  By the addition
    theorem for Legendre polynomials both the far-field pair (P2M then M2P)
    and the near-field pair (P2L then L2P) give exactly the truncated series
        sum_{n <= p} r_<^n / r_>^(n+1) P_n(cos g),
    r_< and r_> the smaller and larger of |s - c| and |y - c|, g the angle
    between s - c and y - c.  A wrong or missing term of any degree changes
    the value by more than the tolerance."""
    from scipy.special import eval_legendre
    c = np.array([0.1, -0.2, 0.3])
    near = c + np.array([0.3, 0.2, -0.25])
    far = c + np.array([-0.9, 0.6, 0.8])
    u, v = near - c, far - c
    rs, rl = np.linalg.norm(u), np.linalg.norm(v)
    cg = u @ v / (rs * rl)
    series = sum(rs ** n / rl ** (n + 1) * eval_legendre(n, cg) for n in range(p + 1))
    phi_far, _ = oracle.m2p(p, c, oracle.p2m(p, c, near[None], [1.0]), far[None])
    phi_near, _ = oracle.l2p(p, c, oracle.p2l(p, c, far[None], [1.0]), near[None])
    assert phi_far[0] == pytest.approx(series, rel=1e-13)
    assert phi_near[0] == pytest.approx(series, rel=1e-13)


def test_p2m_m2p_error_decreases_geometrically():
    rng = np.random.default_rng(2)
    c = np.zeros(3)
    src = _cluster(rng, c, 1.0, 60)
    q = rng.uniform(-1, 1, 60)
    tgt = np.array([[2.5, 0.4, -0.3], [0.2, -2.2, 1.0]])
    pd, gd = oracle.direct(src, q, tgt)
    errs = []
    for p in range(2, 16, 2):
        phi, g = oracle.m2p(p, c, oracle.p2m(p, c, src, q), tgt)
        errs.append(max(np.abs(phi - pd).max() / np.abs(pd).max(), np.abs(g - gd).max() / np.abs(gd).max()))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6


def test_m2m_is_exact_reexpansion():
    """M2M(P2M(children)) == P2M(parent) at degree <= p (no truncation)."""
    p = 10
    rng = np.random.default_rng(3)
    cp = np.array([0.5, 0.5, 0.5])
    Mp_direct = np.zeros((p + 1) ** 2, complex)
    Mp_m2m = np.zeros((p + 1) ** 2, complex)
    for o in range(8):
        h = np.array([(o >> 0) & 1, (o >> 1) & 1, (o >> 2) & 1]) - 0.5
        cc = cp + 0.5 * h
        pts = _cluster(rng, cc, 0.5, 20)
        q = rng.uniform(-1, 1, 20)
        Mp_direct += oracle.p2m(p, cp, pts, q)
        Mp_m2m += oracle.m2m(p, cc, oracle.p2m(p, cc, pts, q), cp)
    np.testing.assert_allclose(Mp_m2m, Mp_direct, rtol=0, atol=1e-13 * np.abs(Mp_direct).max())


def test_l2l_is_exact_recentering():
    """L2P(L2L(L)) == L2P(L): a truncated local expansion is a polynomial."""
    p = 10
    rng = np.random.default_rng(4)
    cp = np.zeros(3)
    src = _cluster(rng, np.array([4.0, 0.0, 1.0]), 1.0, 30)
    q = rng.uniform(-1, 1, 30)
    L = oracle.p2l(p, cp, src, q)
    cc = cp + np.array([0.25, -0.25, 0.25])
    Lc = oracle.l2l(p, cp, L, cc)
    tgt = _cluster(rng, cc, 0.5, 20)
    a, ga = oracle.l2p(p, cp, L, tgt)
    b, gb = oracle.l2p(p, cc, Lc, tgt)
    np.testing.assert_allclose(b, a, rtol=1e-13)
    np.testing.assert_allclose(gb, ga, rtol=1e-11, atol=1e-13 * np.abs(ga).max())


@pytest.mark.parametrize("p", [4, 8, 12])
def test_m2l_then_l2p_matches_direct(p):
    """Well-separated boxes (centres 2 box sides apart): M2L+L2P approaches
    the direct sum, error shrinking with p, and P2L+L2P agrees likewise."""
    rng = np.random.default_rng(10 + p)
    cA = np.array([0.0, 0.0, 0.0])
    cB = np.array([2.0, 1.0, -2.0])
    src = _cluster(rng, cA, 1.0, 50)
    q = rng.uniform(-1, 1, 50)
    tgt = _cluster(rng, cB, 1.0, 50)
    pd, gd = oracle.direct(src, q, tgt)
    L = oracle.m2l(p, cA, oracle.p2m(p, cA, src, q), cB)
    phi, g = oracle.l2p(p, cB, L, tgt)
    tol, gtol = {4: (3e-3, 3e-2), 8: (3e-6, 1e-4), 12: (1e-8, 1e-6)}[p]
    assert np.linalg.norm(phi - pd) / np.linalg.norm(pd) < tol
    assert np.linalg.norm(g - gd) / np.linalg.norm(gd) < gtol
    L2 = oracle.p2l(p, cB, src, q)
    phi2, _ = oracle.l2p(p, cB, L2, tgt)
    assert np.linalg.norm(phi2 - pd) / np.linalg.norm(pd) < tol


def test_m2l_transpose_symmetry():
    """Pairing a multipole of A with a local of B through M2L is symmetric:
    conj-pairing <N_B, M2L(A->B) M_A> with R-moments equals the same with
    A and B swapped.  Concretely the potential at y from x via
    P2M(x)->M2L->L2P equals the potential at x from y (kernel symmetry of the
    truncated operator)."""
    p = 8
    cA = np.array([0.0, 0.0, 0.0])
    cB = np.array([2.0, -3.0, 2.0])
    x = cA + np.array([0.21, -0.33, 0.12])
    y = cB + np.array([-0.4, 0.05, 0.3])
    k_xy = oracle.l2p(p, cB, oracle.m2l(p, cA, oracle.p2m(p, cA, x[None], [1.0]), cB), y[None])[0][0]
    k_yx = oracle.l2p(p, cA, oracle.m2l(p, cB, oracle.p2m(p, cB, y[None], [1.0]), cA), x[None])[0][0]
    assert k_xy == pytest.approx(k_yx, rel=1e-14)
    assert k_xy == pytest.approx(1 / np.linalg.norm(x - y), rel=1e-3)


def test_expansion_gradients_match_fd():
    """Gradients of L2P and M2P are derivatives of the evaluated expansions."""
    p = 9
    rng = np.random.default_rng(7)
    c = np.array([0.3, 0.1, -0.2])
    src = _cluster(rng, c + np.array([3.0, 0, 0]), 1.0, 10)
    q = rng.uniform(-1, 1, 10)
    L = oracle.p2l(p, c, src, q)
    M = oracle.p2m(p, c + np.array([3.0, 0, 0]), src, q)
    h = 1e-5
    for fn, X, cc in ((oracle.l2p, L, c), (oracle.m2p, M, c + np.array([3.0, 0, 0]))):
        x0 = c + np.array([0.2, -0.1, 0.15])
        _, g = fn(p, cc, X, x0[None])
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fp = fn(p, cc, X, (x0 + e)[None])[0][0]
            fm = fn(p, cc, X, (x0 - e)[None])[0][0]
            assert (fp - fm) / (2 * h) == pytest.approx(g[0, a], rel=1e-7, abs=1e-9)

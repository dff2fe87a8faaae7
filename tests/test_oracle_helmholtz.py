"""Pins of the Helmholtz oracle (kernel e^{i kappa r}/r) against what the
mathematics fixes: library special functions, exact quadrature, exact Gaunt
coefficients, the addition theorems against direct evaluation, and the FMM
against the direct sum.  None of these re-types an oracle formula."""
import numpy as np
import pytest
import scipy.special as sp

import oracle

KAPPA = 7.0  # the wave number of the paper's Helmholtz preconditioning test (§4.2)


@pytest.mark.parametrize("x", [1e-6, 1e-3, 0.3, 0.99, 1.0, 2.5, np.pi, 7.0, 17.3, 40.0])
def test_spherical_bessel_matches_scipy(x):
    j, y = oracle.sph_bessel(30, x)
    for n in range(31):
        jr, yr = sp.spherical_jn(n, x), sp.spherical_yn(n, x)
        # near a zero of j_n only absolute accuracy (on the scale 1/x) is defined
        assert abs(j[n] - jr) <= 1e-13 * max(abs(jr), min(1.0, 1.0 / x) * 1e-3), (n, j[n], jr)
        assert abs(y[n] - yr) <= 1e-13 * abs(yr), (n, y[n], yr)


def test_spherical_bessel_wronskian():
    # j_n y_{n-1} - j_{n-1} y_n = 1/x^2 (a closed form independent of any routine)
    for x in (0.5, 3.0, 11.0):
        j, y = oracle.sph_bessel(20, x)
        for n in range(1, 21):
            w = j[n] * y[n - 1] - j[n - 1] * y[n]
            assert abs(w * x * x - 1.0) < 1e-10


def test_spherical_harmonics_match_scipy():
    rng = np.random.default_rng(1)
    for _ in range(12):
        x = rng.normal(size=3)
        r = np.linalg.norm(x)
        th, ph = np.arccos(x[2] / r), np.arctan2(x[1], x[0])
        Y = oracle.sph_harmonics(12, x)
        for n in range(13):
            for m in range(-n, n + 1):
                assert abs(Y[n * n + n + m] - sp.sph_harm_y(n, m, th, ph)) < 1e-13


def test_spherical_harmonics_on_the_pole_and_orthonormality():
    Y = oracle.sph_harmonics(6, [0.0, 0.0, 0.0])  # taken as the +z direction
    for n in range(7):
        assert abs(Y[n * n + n] - np.sqrt((2 * n + 1) / (4 * np.pi))) < 1e-14
        for m in range(1, n + 1):
            assert Y[n * n + n + m] == 0 and Y[n * n + n - m] == 0
    # orthonormality by a product rule exact at this degree
    xs, ws = oracle.gauss_legendre(12)
    nphi = 25
    gram = np.zeros((49, 49), complex)
    for u, w in zip(xs, ws):
        s = np.sqrt(1 - u * u)
        for k in range(nphi):
            f = 2 * np.pi * k / nphi
            Y = oracle.sph_harmonics(6, [s * np.cos(f), s * np.sin(f), u])
            gram += w * (2 * np.pi / nphi) * np.outer(Y, np.conj(Y))
    assert np.max(np.abs(gram - np.eye(49))) < 1e-13


def test_gauss_legendre_is_exact_to_degree_2n_minus_1():
    for n in (1, 2, 5, 18):
        x, w = oracle.gauss_legendre(n)
        for k in range(2 * n):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs(np.sum(w * x ** k) - exact) < 1e-14


def test_gaunt_coefficients_match_sympy_exactly():
    wigner = pytest.importorskip("sympy.physics.wigner")
    p = 4
    G = oracle.gaunt_table(p)
    worst = 0.0
    for n in range(p + 1):
        for m in range(-n, n + 1):
            for n2 in range(p + 1):
                for m2 in range(-n2, n2 + 1):
                    for l in range(abs(n - n2), n + n2 + 1):
                        mu = m - m2
                        if abs(mu) > l:
                            continue
                        # int Y_n^m conj(Y_n2^m2) conj(Y_l^mu) with conj(Y_l^m) = (-1)^m Y_l^-m
                        ref = (-1) ** m * float(wigner.gaunt(n, n2, l, m, -m2, -mu))
                        worst = max(worst, abs(oracle.gaunt(G, p, n, m, n2, m2, l) - ref))
    assert worst < 1e-14


def test_addition_theorem_of_the_kernel():
    x = np.array([0.4, -0.3, 0.5])
    y = np.array([0.05, 0.1, -0.08])
    r = np.linalg.norm(x - y)
    exact = np.exp(1j * KAPPA * r) / r
    S = oracle.h_wave(24, KAPPA, x, 1)
    R = oracle.h_wave(24, KAPPA, y, 0)
    assert abs(4 * np.pi * 1j * KAPPA * np.sum(S * np.conj(R)) - exact) < 1e-13


@pytest.mark.parametrize("kind", ["RR", "SR", "SS"])
def test_translation_coefficients_reproduce_shifted_wave_functions(kind):
    """R_n^m(x+t) = sum (R|R)(t) R(x); S_n^m(x+t) = sum (S|R)(t) R(x) for |x|<|t|;
    S_n^m(x+t) = sum (R|R)(t) S(x) for |x|>|t| -- against direct evaluation, with
    the error falling geometrically in the truncation degree."""
    small, large = np.array([0.05, -0.04, 0.06]), np.array([0.3, 0.25, -0.35])
    xs, t = (small, np.array([0.1, 0.2, -0.15])) if kind == "RR" else \
        (small, large) if kind == "SR" else (large, small)
    errs = []
    for P in (6, 20):
        G = oracle.gaunt_table(P)
        worst = 0.0
        for n in range(3):
            for m in range(-n, n + 1):
                e = np.zeros((P + 1) ** 2, complex)
                e[n * n + n + m] = 1.0
                col = oracle.h_translate(P, KAPPA, G, t, 1 if kind == "SR" else 0, e)
                ref = oracle.h_wave(P, KAPPA, xs + t, 0 if kind == "RR" else 1)[n * n + n + m]
                basis = oracle.h_wave(P, KAPPA, xs, 1 if kind == "SS" else 0)
                worst = max(worst, abs(np.sum(col * basis) - ref) / abs(ref))
        errs.append(worst)
    assert errs[1] < 1e-10 and errs[1] < errs[0] * 1e-2, errs


def _cluster(rng, c, r, n):
    return np.asarray(c) + rng.uniform(-r, r, size=(n, 3))


def test_p2m_m2p_and_p2l_l2p_converge_to_the_direct_sum():
    rng = np.random.default_rng(5)
    src = _cluster(rng, [0, 0, 0], 0.1, 30)
    q = rng.normal(size=30) + 1j * rng.normal(size=30)
    far = _cluster(rng, [0.9, -0.5, 0.4], 0.1, 20)
    ref = oracle.h_direct(src, q, KAPPA, far)
    e = []
    for p in (6, 12):
        M = oracle.h_p2m(p, KAPPA, [0, 0, 0], src, q)
        e.append(np.max(np.abs(oracle.h_m2p(p, KAPPA, [0, 0, 0], M, far) - ref)) / np.max(np.abs(ref)))
        L = oracle.h_p2l(p, KAPPA, [0.9, -0.5, 0.4], src, q)
        e.append(np.max(np.abs(oracle.h_l2p(p, KAPPA, [0.9, -0.5, 0.4], L, far) - ref)) /
                 np.max(np.abs(ref)))
    assert e[2] < 1e-9 and e[3] < 1e-9 and e[2] < e[0] and e[3] < e[1], e


def test_m2m_m2l_l2l_chain_converges_to_the_direct_sum():
    rng = np.random.default_rng(6)
    cs, cp = np.array([0.05, 0.05, 0.05]), np.zeros(3)  # child and parent source centres
    tp, tc = np.array([1.0, 0.6, -0.8]), np.array([1.05, 0.55, -0.75])
    src = _cluster(rng, cs, 0.05, 25)
    q = rng.normal(size=25) + 1j * rng.normal(size=25)
    tgt = _cluster(rng, tc, 0.05, 15)
    ref = oracle.h_direct(src, q, KAPPA, tgt)
    errs = []
    for p in (6, 10, 14):
        G = oracle.gaunt_table(p)
        M = oracle.h_m2m(p, KAPPA, G, cs, oracle.h_p2m(p, KAPPA, cs, src, q), cp)
        L = oracle.h_l2l(p, KAPPA, G, tp, oracle.h_m2l(p, KAPPA, G, cp, M, tp), tc)
        errs.append(np.max(np.abs(oracle.h_l2p(p, KAPPA, tc, L, tgt) - ref)) / np.max(np.abs(ref)))
    assert errs[2] < 1e-8 and errs[0] > errs[1] > errs[2], errs


def test_direct_sum_closed_forms():
    # two charges: phi_0 = q_1 e^{i k r}/r; the small-kappa limit is the Laplace sum
    src = np.array([[0.0, 0, 0], [0.3, 0.4, 0.0]])
    q = np.array([1.0 + 2j, -0.5 + 0.25j])
    phi = oracle.h_direct(src, q, KAPPA)
    assert abs(phi[0] - q[1] * np.exp(1j * KAPPA * 0.5) / 0.5) < 1e-14
    assert abs(phi[1] - q[0] * np.exp(1j * KAPPA * 0.5) / 0.5) < 1e-14
    rng = np.random.default_rng(7)
    x = rng.uniform(size=(50, 3))
    qr = rng.normal(size=50)
    lap = oracle.direct(x, qr, grad=False)
    lap = lap[0] if isinstance(lap, tuple) else lap
    hel = oracle.h_direct(x, qr, 1e-9)
    assert np.max(np.abs(hel.real - lap)) < 1e-12 * np.max(np.abs(lap))


@pytest.mark.parametrize("dist", ["cube", "plummer"])
def test_fmm_converges_to_the_direct_sum_and_is_complex_symmetric(dist):
    from paper_1602_02244_gb300 import workloads
    n = 1500
    # the low-frequency expansions need kappa x (box side) of order one at level 2:
    # the Plummer sphere is scaled into a cube of side ~2, like [-1, 1]^3
    x = workloads.uniform_cube(n, seed=11) if dist == "cube" else \
        workloads.plummer(n, seed=11) / 10.0
    rng = np.random.default_rng(12)
    q = rng.normal(size=n) + 1j * rng.normal(size=n)
    t = oracle.Tree(x, 24)
    if dist == "plummer":
        assert len(t.w_idx) > 0 and len(t.x_idx) > 0
    ref = oracle.h_direct(x, q, KAPPA)
    errs = [np.linalg.norm(t.helmholtz_eval(p, KAPPA, q) - ref) / np.linalg.norm(ref)
            for p in (4, 8, 12)]
    assert errs[2] < 1e-6 and errs[0] > errs[1] > errs[2], errs
    # the Helmholtz matrix is complex symmetric: e_a^T A e_b = e_b^T A e_a
    a, b = 3, 1000
    ea = np.zeros(n, complex)
    eb = np.zeros(n, complex)
    ea[a] = eb[b] = 1.0
    Aab = t.helmholtz_eval(12, KAPPA, eb)[a]
    Aba = t.helmholtz_eval(12, KAPPA, ea)[b]
    r = np.linalg.norm(x[a] - x[b])
    assert abs(Aab - Aba) < 1e-6 * abs(Aab)
    assert abs(Aab - np.exp(1j * KAPPA * r) / r) < 1e-5 * abs(Aab)

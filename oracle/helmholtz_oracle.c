/*
 * helmholtz_oracle.c -- plain FP64 CPU oracle for the FMM mat-vec with the
 * Helmholtz kernel e^{i kappa r} / r (the paper's second kernel: §1 compares
 * FMM and HSS "for Laplace and Helmholtz kernels", and §4.2 preconditions the
 * Helmholtz equation with wave number kappa = 7 on [-1, 1]^3).
 *
 * TEST INFRASTRUCTURE ONLY (see fmm_oracle.h): the GPU library shares no
 * code, header, table or constant with it.  Plain loops in the order of the
 * definitions; OpenMP only splits independent boxes of one pass.
 *
 * The paper prints no expansion formula.  This oracle takes the textbook
 * low-frequency expansions (Gegenbauer's addition theorem):
 *   Y_n^m(t, f) = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m(cos t) e^{i m f},
 *                 P_n^m with the Condon-Shortley phase, Y_n^{-m} = (-1)^m conj(Y_n^m);
 *   j_n, y_n the spherical Bessel functions, h_n = j_n + i y_n;
 *   R_n^m(x) = j_n(kappa|x|) Y_n^m(x/|x|),  S_n^m(x) = h_n(kappa|x|) Y_n^m(x/|x|).
 *   For |y| < |x|:
 *     e^{i kappa |x-y|} / |x-y| = 4 pi i kappa sum_{n,m} S_n^m(x) conj(R_n^m(y))
 *                               = 4 pi i kappa sum_{n,m} R_n^m(y) h_n(kappa|x|) conj(Y_n^m(x^)).
 * Multipole about c: phi(x) = sum M_n^m S_n^m(x - c),
 *   P2M: M_n^m += 4 pi i kappa q conj(R_n^m(y - c)).
 * Local about c: phi(x) = sum L_n^m R_n^m(x - c),
 *   P2L: L_n^m += 4 pi i kappa q h_n(kappa|y - c|) conj(Y_n^m((y - c)^)).
 * Translations, with the Gaunt coefficient
 *   G(n,m; n',m'; l) = integral over the sphere of Y_n^m conj(Y_n'^m') conj(Y_l^{m-m'}),
 * and the translation coefficients (plane-wave expansion of R_n^m(x + t))
 *   (X|R)_{n'n}^{m'm}(t) = 4 pi sum_l i^{n'+l-n} X_l^{m-m'}(t) G(n,m; n',m'; l),  X = R or S:
 *   R_n^m(x + t) = sum_{n',m'} (R|R)_{n'n}^{m'm}(t) R_n'^m'(x)               (all x, t)
 *   S_n^m(x + t) = sum_{n',m'} (S|R)_{n'n}^{m'm}(t) R_n'^m'(x)               (|x| < |t|)
 *   S_n^m(x + t) = sum_{n',m'} (R|R)_{n'n}^{m'm}(t) S_n'^m'(x)               (|x| > |t|)
 * so that, with every sum truncated at degree p,
 *   M2M  M'(c2)  = (R|R)(c2 - c1) M(c1),
 *   M2L  L(c2)  += (S|R)(c2 - c1) M(c1),
 *   L2L  L'(c2)  = (R|R)(c2 - c1) L(c1).
 * Each identity is pinned by the tests against direct evaluation.
 *
 * Complex arrays hold (p+1)^2 entries, index n*n+n+m, as interleaved (re, im).
 */
#include "fmm_oracle.h"
#include "oracle_tree.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static inline int hidx(int n, int m) { return n * n + n + m; }
static inline int hncoef(int p) { return (p + 1) * (p + 1); }

static const double kPi = 3.14159265358979323846;

/* ------------------------------------------------------------------------
 * Spherical Bessel functions j_n(x), y_n(x), n = 0..nmax.
 *  - x < 1: the power series
 *      j_n(x) = x^n / (2n+1)!! sum_k (-x^2/2)^k / (k! (2n+3)(2n+5)...(2n+2k+1)),
 *    whose terms fall monotonically for x < 1.
 *  - x >= 1: Miller's algorithm.  The recurrence f_{n-1} = (2n+1)/x f_n - f_{n+1}
 *    is run downwards from f_{N+1} = 0, f_N = 1 with N far above nmax and x,
 *    and the result scaled to j_0 = sin x / x or j_1 = sin x / x^2 - cos x / x,
 *    whichever is larger in magnitude (their zeros interlace).
 *  - y_n by the upward recurrence y_{n+1} = (2n+1)/x y_n - y_{n-1} from
 *    y_0 = -cos x / x, y_1 = -cos x / x^2 - sin x / x (stable upwards).
 * x = 0: j_0 = 1, j_n = 0 for n > 0; y is not defined there (left untouched).
 * ---------------------------------------------------------------------- */
void oracle_sph_bessel(int nmax, double x, double *j, double *y) {
  if (x == 0.0) {
    for (int n = 0; n <= nmax; ++n) j[n] = n == 0 ? 1.0 : 0.0;
    return;
  }
  if (x < 1.0) {
    double lead = 1.0; /* x^n / (2n+1)!! */
    for (int n = 0; n <= nmax; ++n) {
      if (n > 0) lead *= x / (2.0 * n + 1.0);
      double sum = 0.0, term = 1.0;
      for (int k = 0; k < 60; ++k) {
        if (k > 0) term *= -0.5 * x * x / ((double)k * (2.0 * n + 2.0 * k + 1.0));
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
      }
      j[n] = lead * sum;
    }
  } else {
    int N = nmax + (int)x + 40;
    double *f = malloc(sizeof(double) * (size_t)(N + 2));
    f[N + 1] = 0.0;
    f[N] = 1.0;
    for (int n = N; n >= 1; --n) {
      f[n - 1] = (2.0 * n + 1.0) / x * f[n] - f[n + 1];
      if (fabs(f[n - 1]) > 1e250) /* keep the recurrence in range */
        for (int k = n - 1; k <= N + 1; ++k) f[k] *= 1e-250;
    }
    double j0 = sin(x) / x, j1 = sin(x) / (x * x) - cos(x) / x;
    double scale = fabs(j0) >= fabs(j1) ? j0 / f[0] : j1 / f[1];
    for (int n = 0; n <= nmax; ++n) j[n] = f[n] * scale;
    free(f);
  }
  if (y) {
    y[0] = -cos(x) / x;
    if (nmax >= 1) y[1] = -cos(x) / (x * x) - sin(x) / x;
    for (int n = 1; n < nmax; ++n) y[n + 1] = (2.0 * n + 1.0) / x * y[n] - y[n - 1];
  }
}

/* ------------------------------------------------------------------------
 * Orthonormal spherical harmonics Y_n^m of the direction of x, n <= p, from
 * their definition: P_n^m(u) (u = cos t) by P_m^m = (-1)^m (2m-1)!! (1-u^2)^{m/2},
 * P_{m+1}^m = (2m+1) u P_m^m, (n-m) P_n^m = (2n-1) u P_{n-1}^m - (n+m-1) P_{n-2}^m;
 * times sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) and e^{i m f}, f = atan2(y, x).
 * x = 0 is taken as the direction of the z axis.
 * ---------------------------------------------------------------------- */
void oracle_sph_harmonics(int p, const double x[3], double *Yout) {
  cplx *Y = (cplx *)Yout;
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double u = r > 0.0 ? x[2] / r : 1.0;
  double s = sqrt(fmax(0.0, 1.0 - u * u));
  double f = (x[0] == 0.0 && x[1] == 0.0) ? 0.0 : atan2(x[1], x[0]);
  for (int m = 0; m <= p; ++m) {
    /* P_m^m */
    double pmm = 1.0;
    for (int k = 1; k <= m; ++k) pmm *= -(2.0 * k - 1.0) * s;
    double pprev = 0.0, pcur = pmm;
    for (int n = m; n <= p; ++n) {
      if (n == m + 1) {
        pprev = pcur;
        pcur = (2.0 * m + 1.0) * u * pmm;
      } else if (n > m + 1) {
        double next = ((2.0 * n - 1.0) * u * pcur - (n + m - 1.0) * pprev) / (double)(n - m);
        pprev = pcur;
        pcur = next;
      }
      double ratio = 1.0; /* (n-m)! / (n+m)! */
      for (int k = n - m + 1; k <= n + m; ++k) ratio /= (double)k;
      double norm = sqrt((2.0 * n + 1.0) / (4.0 * kPi) * ratio);
      Y[hidx(n, m)] = norm * pcur * cexp(I * (double)m * f);
      if (m > 0) Y[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(Y[hidx(n, m)]);
    }
  }
}

/* R_n^m(x) (singular = 0) or S_n^m(x) (singular = 1), n <= p */
void oracle_h_wave(int p, double kappa, const double x[3], int singular, double *Xout) {
  cplx *X = (cplx *)Xout;
  double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double *j = malloc(sizeof(double) * (size_t)(p + 1));
  double *y = malloc(sizeof(double) * (size_t)(p + 1));
  cplx *Y = malloc(sizeof(cplx) * (size_t)hncoef(p));
  oracle_sph_bessel(p, kappa * r, j, singular ? y : NULL);
  oracle_sph_harmonics(p, x, (double *)Y);
  for (int n = 0; n <= p; ++n) {
    cplx radial = singular ? j[n] + I * y[n] : j[n];
    for (int m = -n; m <= n; ++m) X[hidx(n, m)] = radial * Y[hidx(n, m)];
  }
  free(j);
  free(y);
  free(Y);
}

/* ------------------------------------------------------------------------
 * Gauss-Legendre rule of n nodes on [-1, 1]: the roots of P_n by Newton's
 * method from cos(pi (k + 3/4) / (n + 1/2)), weights 2 / ((1 - x^2) P_n'(x)^2).
 * Exact for polynomials of degree <= 2n - 1.
 * ---------------------------------------------------------------------- */
void oracle_gauss_legendre(int n, double *xs, double *ws) {
  for (int k = 0; k < n; ++k) {
    double x = cos(kPi * (k + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x; /* P_0, P_1, then up to P_n */
      for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (x * p1 - p0) / (x * x - 1.0); /* P_n'(x) */
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    /* recompute the derivative at the converged node */
    double p0 = 1.0, p1 = x;
    for (int m = 2; m <= n; ++m) {
      double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    xs[k] = x;
    ws[k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

/* ------------------------------------------------------------------------
 * Gaunt coefficients G(n,m; n',m'; l) = integral of Y_n^m conj(Y_n'^m')
 * conj(Y_l^mu) over the unit sphere, mu = m - m' (other mu give zero: the
 * azimuthal integral of e^{i(m - m' - mu) f} is 2 pi delta).  With
 * Y_n^m(t, f) = Y_n^m(t, 0) e^{i m f} the integral is
 *   2 pi * integral_{-1}^{1} Y_n^m(t,0) Y_n'^m'(t,0) Y_l^mu(t,0) d(cos t),
 * a polynomial of degree n + n' + l <= 4p in cos t (the powers of sin t pair
 * up), integrated exactly by 2p + 2 Gauss-Legendre nodes.
 * Table layout for n, n' <= p: entry ((hidx(n,m) * NC + hidx(n',m')) * (p+1)
 * + (l - |n - n'|)/2) for l = |n-n'|, |n-n'|+2, ..., n+n'.
 * ---------------------------------------------------------------------- */
int64_t oracle_gaunt_size(int p) { return (int64_t)hncoef(p) * hncoef(p) * (p + 1); }

void oracle_gaunt_table(int p, double *G) {
  int nq = 2 * p + 2, P2 = 2 * p, NC = hncoef(p), N2 = hncoef(P2);
  double *xs = malloc(sizeof(double) * nq), *ws = malloc(sizeof(double) * nq);
  oracle_gauss_legendre(nq, xs, ws);
  /* Y_n^m(t_k, 0), n <= 2p, real (f = 0) */
  double *T = malloc(sizeof(double) * (size_t)nq * N2);
  cplx *Y = malloc(sizeof(cplx) * (size_t)N2);
  for (int k = 0; k < nq; ++k) {
    double dir[3] = {sqrt(fmax(0.0, 1.0 - xs[k] * xs[k])), 0.0, xs[k]};
    oracle_sph_harmonics(P2, dir, (double *)Y);
    for (int c = 0; c < N2; ++c) T[(size_t)k * N2 + c] = creal(Y[c]);
  }
  memset(G, 0, sizeof(double) * (size_t)oracle_gaunt_size(p));
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m)
      for (int n2 = 0; n2 <= p; ++n2)
        for (int m2 = -n2; m2 <= n2; ++m2) {
          int mu = m - m2, l0 = abs(n - n2);
          for (int l = l0; l <= n + n2; l += 2) {
            if (abs(mu) > l) continue;
            double s = 0.0;
            for (int k = 0; k < nq; ++k)
              s += ws[k] * T[(size_t)k * N2 + hidx(n, m)] * T[(size_t)k * N2 + hidx(n2, m2)] *
                   T[(size_t)k * N2 + hidx(l, mu)];
            G[((size_t)hidx(n, m) * NC + hidx(n2, m2)) * (p + 1) + (l - l0) / 2] = 2.0 * kPi * s;
          }
        }
  free(xs);
  free(ws);
  free(T);
  free(Y);
}

/* out[n',m'] += sum_{n,m} (X|R)_{n'n}^{m'm}(t) in[n,m] for n, n' <= p, with
 * X = S (singular = 1: M2L) or R (singular = 0: M2M, L2L); G from
 * oracle_gaunt_table(p). */
void oracle_h_translate(int p, double kappa, const double *G, const double t[3], int singular,
                        const double *in_, double *out_) {
  const cplx *in = (const cplx *)in_;
  cplx *out = (cplx *)out_;
  int NC = hncoef(p);
  cplx *X = malloc(sizeof(cplx) * (size_t)hncoef(2 * p));
  oracle_h_wave(2 * p, kappa, t, singular, (double *)X);
  for (int n2 = 0; n2 <= p; ++n2)
    for (int m2 = -n2; m2 <= n2; ++m2) {
      cplx acc = 0.0;
      for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
          int mu = m - m2, l0 = abs(n - n2);
          cplx coef = 0.0;
          for (int l = l0; l <= n + n2; l += 2) {
            if (abs(mu) > l) continue;
            /* i^{n'+l-n}: the exponent is even, so this is +-1 */
            double phase = (((n2 + l - n) / 2) & 1) ? -1.0 : 1.0;
            coef += phase * X[hidx(l, mu)] *
                    G[((size_t)hidx(n, m) * NC + hidx(n2, m2)) * (p + 1) + (l - l0) / 2];
          }
          acc += 4.0 * kPi * coef * in[hidx(n, m)];
        }
      out[hidx(n2, m2)] += acc;
    }
  free(X);
}

static void sub3(const double a[3], const double b[3], double d[3]) {
  d[0] = a[0] - b[0];
  d[1] = a[1] - b[1];
  d[2] = a[2] - b[2];
}

void oracle_h_m2m(int p, double kappa, const double *G, const double c_child[3],
                  const double *Mc, const double c_parent[3], double *Mp) {
  double t[3];
  sub3(c_parent, c_child, t);
  oracle_h_translate(p, kappa, G, t, 0, Mc, Mp);
}

void oracle_h_m2l(int p, double kappa, const double *G, const double c_src[3], const double *M,
                  const double c_tgt[3], double *L) {
  double t[3];
  sub3(c_tgt, c_src, t);
  oracle_h_translate(p, kappa, G, t, 1, M, L);
}

void oracle_h_l2l(int p, double kappa, const double *G, const double c_parent[3],
                  const double *Lp, const double c_child[3], double *Lc) {
  double t[3];
  sub3(c_child, c_parent, t);
  oracle_h_translate(p, kappa, G, t, 0, Lp, Lc);
}

/* ------------------------------------------------------------------------
 * Point operations.  q, phi, M, L complex (interleaved); xyz absolute.
 * ---------------------------------------------------------------------- */
void oracle_h_direct(int64_t ns, const double *src, const double *q_, int64_t nt,
                     const double *tgt, double kappa, double *phi_) {
  const cplx *q = (const cplx *)q_;
  cplx *phi = (cplx *)phi_;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nt; ++i) {
    cplx acc = 0.0;
    for (int64_t j = 0; j < ns; ++j) {
      double dx = tgt[3 * i] - src[3 * j], dy = tgt[3 * i + 1] - src[3 * j + 1],
             dz = tgt[3 * i + 2] - src[3 * j + 2];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r == 0.0) continue;
      acc += q[j] * cexp(I * kappa * r) / r;
    }
    phi[i] = acc;
  }
}

void oracle_h_p2m(int p, double kappa, const double c[3], int64_t n, const double *xyz,
                  const double *q_, double *M_) {
  const cplx *q = (const cplx *)q_;
  cplx *M = (cplx *)M_;
  cplx *R = malloc(sizeof(cplx) * (size_t)hncoef(p));
  for (int64_t j = 0; j < n; ++j) {
    double d[3];
    sub3(xyz + 3 * j, c, d);
    oracle_h_wave(p, kappa, d, 0, (double *)R);
    for (int k = 0; k < hncoef(p); ++k) M[k] += 4.0 * kPi * I * kappa * q[j] * conj(R[k]);
  }
  free(R);
}

void oracle_h_p2l(int p, double kappa, const double c[3], int64_t n, const double *xyz,
                  const double *q_, double *L_) {
  const cplx *q = (const cplx *)q_;
  cplx *L = (cplx *)L_;
  double *jn = malloc(sizeof(double) * (size_t)(p + 1));
  double *yn = malloc(sizeof(double) * (size_t)(p + 1));
  cplx *Y = malloc(sizeof(cplx) * (size_t)hncoef(p));
  for (int64_t j = 0; j < n; ++j) {
    double d[3];
    sub3(xyz + 3 * j, c, d);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    oracle_sph_bessel(p, kappa * r, jn, yn);
    oracle_sph_harmonics(p, d, (double *)Y);
    for (int nn = 0; nn <= p; ++nn)
      for (int m = -nn; m <= nn; ++m)
        L[hidx(nn, m)] += 4.0 * kPi * I * kappa * q[j] * (jn[nn] + I * yn[nn]) * conj(Y[hidx(nn, m)]);
  }
  free(jn);
  free(yn);
  free(Y);
}

/* phi[i] += sum_{n,m} C_n^m X_n^m(x_i - c): L2P with X = R, M2P with X = S */
static void h_evaluate(int p, double kappa, const double c[3], const cplx *C, int singular,
                       int64_t n, const double *xyz, cplx *phi) {
  cplx *X = malloc(sizeof(cplx) * (size_t)hncoef(p));
  for (int64_t i = 0; i < n; ++i) {
    double d[3];
    sub3(xyz + 3 * i, c, d);
    oracle_h_wave(p, kappa, d, singular, (double *)X);
    cplx acc = 0.0;
    for (int k = 0; k < hncoef(p); ++k) acc += C[k] * X[k];
    phi[i] += acc;
  }
  free(X);
}

void oracle_h_l2p(int p, double kappa, const double c[3], const double *L, int64_t n,
                  const double *xyz, double *phi) {
  h_evaluate(p, kappa, c, (const cplx *)L, 0, n, xyz, (cplx *)phi);
}

void oracle_h_m2p(int p, double kappa, const double c[3], const double *M, int64_t n,
                  const double *xyz, double *phi) {
  h_evaluate(p, kappa, c, (const cplx *)M, 1, n, xyz, (cplx *)phi);
}

/* ------------------------------------------------------------------------
 * FMM mat-vec with the Helmholtz kernel on a built tree: the pass order and
 * lists of the Laplace oracle (P2M at the leaves, M2M upwards, M2L over V and
 * P2L over X at levels >= 2, L2L downwards, L2P + M2P over W + P2P over U at
 * the leaves).  q and phi complex, in the caller's order.
 * ---------------------------------------------------------------------- */
void oracle_h_fmm_eval(const oracle_tree *t, int p, double kappa, const double *q_in,
                       double *phi_out) {
  int64_t n = t->n, nb = t->nboxes;
  int nc = hncoef(p);
  if (n == 0) return;
  const cplx *qi = (const cplx *)q_in;
  cplx *q = malloc(sizeof(cplx) * n);
  for (int64_t i = 0; i < n; ++i) q[i] = qi[t->perm[i]];
  double *G = malloc(sizeof(double) * (size_t)oracle_gaunt_size(p));
  oracle_gaunt_table(p, G);
  cplx *M = calloc((size_t)nb * nc, sizeof(cplx));
  cplx *L = calloc((size_t)nb * nc, sizeof(cplx));
  cplx *phi = calloc(n, sizeof(cplx));

#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < nb; ++b)
    if (t->box_nchild[b] == 0)
      oracle_h_p2m(p, kappa, t->center[b], t->box_count[b],
                   t->xyz + 3 * (int64_t)t->box_first[b], (const double *)(q + t->box_first[b]),
                   (double *)(M + (size_t)b * nc));
  for (int l = t->nlevels - 2; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = t->level_offset[l]; b < t->level_offset[l + 1]; ++b)
      for (int c = 0; c < t->box_nchild[b]; ++c) {
        int32_t C = t->box_child[b] + c;
        oracle_h_m2m(p, kappa, G, t->center[C], (double *)(M + (size_t)C * nc), t->center[b],
                     (double *)(M + (size_t)b * nc));
      }
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t b = 0; b < nb; ++b) {
    if (t->box_level[b] < 2) continue;
    for (int64_t k = 0; k < t->V[b].n; ++k) {
      int32_t A = t->V[b].a[k];
      oracle_h_m2l(p, kappa, G, t->center[A], (double *)(M + (size_t)A * nc), t->center[b],
                   (double *)(L + (size_t)b * nc));
    }
    for (int64_t k = 0; k < t->X[b].n; ++k) {
      int32_t A = t->X[b].a[k];
      oracle_h_p2l(p, kappa, t->center[b], t->box_count[A],
                   t->xyz + 3 * (int64_t)t->box_first[A], (const double *)(q + t->box_first[A]),
                   (double *)(L + (size_t)b * nc));
    }
  }
  for (int l = 3; l < t->nlevels; ++l) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t b = t->level_offset[l]; b < t->level_offset[l + 1]; ++b) {
      int32_t P = t->box_parent[b];
      oracle_h_l2l(p, kappa, G, t->center[P], (double *)(L + (size_t)P * nc), t->center[b],
                   (double *)(L + (size_t)b * nc));
    }
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t b = 0; b < nb; ++b) {
    if (t->box_nchild[b] != 0) continue;
    int64_t f = t->box_first[b], cnt = t->box_count[b];
    const double *tx = t->xyz + 3 * f;
    if (t->box_level[b] >= 2)
      h_evaluate(p, kappa, t->center[b], L + (size_t)b * nc, 0, cnt, tx, phi + f);
    for (int64_t k = 0; k < t->W[b].n; ++k) {
      int32_t A = t->W[b].a[k];
      h_evaluate(p, kappa, t->center[A], M + (size_t)A * nc, 1, cnt, tx, phi + f);
    }
    for (int64_t k = 0; k < t->U[b].n; ++k) {
      int32_t A = t->U[b].a[k];
      int64_t fa = t->box_first[A], ca = t->box_count[A];
      for (int64_t i = 0; i < cnt; ++i)
        for (int64_t j = fa; j < fa + ca; ++j) {
          double dx = tx[3 * i] - t->xyz[3 * j], dy = tx[3 * i + 1] - t->xyz[3 * j + 1],
                 dz = tx[3 * i + 2] - t->xyz[3 * j + 2];
          double r = sqrt(dx * dx + dy * dy + dz * dz);
          if (r == 0.0) continue;
          phi[f + i] += q[j] * cexp(I * kappa * r) / r;
        }
    }
  }
  cplx *po = (cplx *)phi_out;
  for (int64_t i = 0; i < n; ++i) po[t->perm[i]] = phi[i];
  free(q);
  free(G);
  free(M);
  free(L);
  free(phi);
}

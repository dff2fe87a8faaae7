/*
 * fmm_oracle.c -- plain FP64 CPU oracle for the 3D Laplace FMM mat-vec.
 *
 * TEST INFRASTRUCTURE ONLY (see fmm_oracle.h).  Written for a reader who
 * checks it against the definitions: no blocking, no fusion, no reordering
 * beyond what the definitions state.  OpenMP only splits independent boxes
 * (or targets) of one pass across threads; each box's arithmetic is the
 * sequential loop written here.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (oracle/build.py).
 */
#include "fmm_oracle.h"
#include "oracle_tree.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define MAXDEPTH 21

static inline int idx(int n, int m) { return n * n + n + m; }
static inline int ncoef(int p) { return (p + 1) * (p + 1); }
static inline double sgn(int m) { return (m & 1) ? -1.0 : 1.0; }

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Solid harmonics.  Recurrences follow from the three-term recurrence of the
 * associated Legendre functions, (n-m) P_n^m = (2n-1) x P_{n-1}^m
 * - (n+m-1) P_{n-2}^m, and P_m^m = (-1)^m (2m-1)!! (1-x^2)^{m/2}, multiplied
 * through by the normalisations of the header:
 *   R_m^m = -(x+iy)/(2m) R_{m-1}^{m-1},
 *   (n^2-m^2) R_n^m = (2n-1) z R_{n-1}^m - r^2 R_{n-2}^m,
 *   I_m^m = -(2m-1)(x+iy)/r^2 I_{m-1}^{m-1},
 *   r^2 I_n^m = (2n-1) z I_{n-1}^m - ((n-1)^2-m^2) I_{n-2}^m.
 * ---------------------------------------------------------------------- */
static void regular_c(int p, const double x[3], cplx *R) {
  double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  cplx w = x[0] + I * x[1];
  R[0] = 1.0;
  for (int m = 1; m <= p; ++m) R[idx(m, m)] = -w / (2.0 * m) * R[idx(m - 1, m - 1)];
  for (int m = 0; m <= p; ++m)
    for (int n = m + 1; n <= p; ++n) {
      cplx a = (2.0 * n - 1.0) * x[2] * R[idx(n - 1, m)];
      cplx b = (n - 2 >= m) ? r2 * R[idx(n - 2, m)] : 0.0;
      R[idx(n, m)] = (a - b) / ((double)(n - m) * (double)(n + m));
    }
  for (int n = 1; n <= p; ++n)
    for (int m = 1; m <= n; ++m) R[idx(n, -m)] = sgn(m) * conj(R[idx(n, m)]);
}

static void irregular_c(int p, const double x[3], cplx *Iv) {
  double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  cplx w = x[0] + I * x[1];
  Iv[0] = 1.0 / sqrt(r2);
  for (int m = 1; m <= p; ++m) Iv[idx(m, m)] = -(2.0 * m - 1.0) * w / r2 * Iv[idx(m - 1, m - 1)];
  for (int m = 0; m <= p; ++m)
    for (int n = m + 1; n <= p; ++n) {
      cplx a = (2.0 * n - 1.0) * x[2] * Iv[idx(n - 1, m)];
      cplx b = (n - 2 >= m) ? ((double)(n - 1) * (n - 1) - (double)m * m) * Iv[idx(n - 2, m)] : 0.0;
      Iv[idx(n, m)] = (a - b) / r2;
    }
  for (int n = 1; n <= p; ++n)
    for (int m = 1; m <= n; ++m) Iv[idx(n, -m)] = sgn(m) * conj(Iv[idx(n, m)]);
}

/* harmonic value with the convention X_n^m = 0 for |m| > n or n < 0 */
static inline cplx at(const cplx *X, int p, int n, int m) {
  if (n < 0 || n > p || m < -n || m > n) return 0.0;
  return X[idx(n, m)];
}

void oracle_regular(int p, const double x[3], double *R) { regular_c(p, x, (cplx *)R); }
void oracle_irregular(int p, const double x[3], double *Iv) { irregular_c(p, x, (cplx *)Iv); }

/* ------------------------------------------------------------------------
 * Direct sum: the Green's-function operator of the dense diagonal blocks
 * (§2.2).  phi(x) = sum_j q_j / |x - x_j|, grad phi(x) = -sum_j q_j
 * (x - x_j) / |x - x_j|^3, pairs at zero distance contribute nothing.
 * ---------------------------------------------------------------------- */
void oracle_direct(int64_t ns, const double *src, const double *q, int64_t nt,
                   const double *tgt, double *phi, double *grad) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nt; ++i) {
    double f = 0, gx = 0, gy = 0, gz = 0;
    for (int64_t j = 0; j < ns; ++j) {
      double dx = tgt[3 * i] - src[3 * j];
      double dy = tgt[3 * i + 1] - src[3 * j + 1];
      double dz = tgt[3 * i + 2] - src[3 * j + 2];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      double r = sqrt(r2);
      f += q[j] / r;
      double s = q[j] / (r2 * r);
      gx -= s * dx;
      gy -= s * dy;
      gz -= s * dz;
    }
    phi[i] = f;
    if (grad) {
      grad[3 * i] = gx;
      grad[3 * i + 1] = gy;
      grad[3 * i + 2] = gz;
    }
  }
}

/* ------------------------------------------------------------------------
 * Translations (Greengard & Rokhlin, cited in §2.1; translation operators of
 * §2.2).  Multipole about c: phi(x) = sum M_n^m I_n^m(x - c).
 * Local about c:            phi(x) = sum L_n^m R_n^m(x - c).
 * ---------------------------------------------------------------------- */

/* P2M: from 1/|x-y| = sum conj(R(y-c)) I(x-c):  M_n^m = sum_j q_j conj(R_n^m(x_j - c)) */
void oracle_p2m(int p, const double c[3], int64_t n, const double *xyz,
                const double *q, double *Mout) {
  cplx *M = (cplx *)Mout;
  cplx *R = malloc(sizeof(cplx) * ncoef(p));
  for (int64_t j = 0; j < n; ++j) {
    double d[3] = {xyz[3 * j] - c[0], xyz[3 * j + 1] - c[1], xyz[3 * j + 2] - c[2]};
    regular_c(p, d, R);
    for (int k = 0; k < ncoef(p); ++k) M[k] += q[j] * conj(R[k]);
  }
  free(R);
}

/* M2M: x_j - c_p = (x_j - c_c) + (c_c - c_p) in the regular addition theorem:
 *      M_n^m(parent) = sum_{k<=n, l} conj(R_{n-k}^{m-l}(c_c - c_p)) M_k^l(child) */
void oracle_m2m(int p, const double cc[3], const double *Mcin, const double cp[3],
                double *Mpout) {
  const cplx *Mc = (const cplx *)Mcin;
  cplx *Mp = (cplx *)Mpout;
  cplx *R = malloc(sizeof(cplx) * ncoef(p));
  double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
  regular_c(p, d, R);
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m) {
      cplx s = 0;
      for (int k = 0; k <= n; ++k)
        for (int l = -k; l <= k; ++l) s += conj(at(R, p, n - k, m - l)) * Mc[idx(k, l)];
      Mp[idx(n, m)] += s;
    }
  free(R);
}

/* M2L: x - c_A = (x - c_B) + d with d = c_B - c_A; the irregular addition
 * theorem plus conj(R_n^m) = (-1)^m R_n^{-m} and phi real give
 *      L_n^m(B) = (-1)^{n+m} sum_{k,l} M_k^l(A) I_{n+k}^{l-m}(d)
 * (degrees up to 2p of I are needed). */
void oracle_m2l(int p, const double cA[3], const double *Min, const double cB[3],
                double *Lout) {
  const cplx *M = (const cplx *)Min;
  cplx *L = (cplx *)Lout;
  int p2 = 2 * p;
  cplx *Iv = malloc(sizeof(cplx) * ncoef(p2));
  double d[3] = {cB[0] - cA[0], cB[1] - cA[1], cB[2] - cA[2]};
  irregular_c(p2, d, Iv);
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m) {
      cplx s = 0;
      for (int k = 0; k <= p; ++k)
        for (int l = -k; l <= k; ++l) s += M[idx(k, l)] * Iv[idx(n + k, l - m)];
      L[idx(n, m)] += sgn(n + m) * s;
    }
  free(Iv);
}

/* L2L: x - c_p = (x - c_c) + (c_c - c_p) in the regular addition theorem:
 *      L_k^l(child) = sum_{n>=k, m} L_n^m(parent) R_{n-k}^{m-l}(c_c - c_p) */
void oracle_l2l(int p, const double cp[3], const double *Lpin, const double cc[3],
                double *Lcout) {
  const cplx *Lp = (const cplx *)Lpin;
  cplx *Lc = (cplx *)Lcout;
  cplx *R = malloc(sizeof(cplx) * ncoef(p));
  double d[3] = {cc[0] - cp[0], cc[1] - cp[1], cc[2] - cp[2]};
  regular_c(p, d, R);
  for (int k = 0; k <= p; ++k)
    for (int l = -k; l <= k; ++l) {
      cplx s = 0;
      for (int n = k; n <= p; ++n)
        for (int m = -n; m <= n; ++m) s += Lp[idx(n, m)] * at(R, p, n - k, m - l);
      Lc[idx(k, l)] += s;
    }
  free(R);
}

/* P2L: 1/|x - y| = sum conj(R(x - c)) I(y - c) for |x - c| < |y - c|, and phi
 * real:  L_n^m = sum_j q_j conj(I_n^m(x_j - c)) */
void oracle_p2l(int p, const double c[3], int64_t n, const double *xyz,
                const double *q, double *Lout) {
  cplx *L = (cplx *)Lout;
  cplx *Iv = malloc(sizeof(cplx) * ncoef(p));
  for (int64_t j = 0; j < n; ++j) {
    double d[3] = {xyz[3 * j] - c[0], xyz[3 * j + 1] - c[1], xyz[3 * j + 2] - c[2]};
    irregular_c(p, d, Iv);
    for (int k = 0; k < ncoef(p); ++k) L[k] += q[j] * conj(Iv[k]);
  }
  free(Iv);
}

/* L2P: phi = sum L_n^m R_n^m(x - c); gradient from the derivative rules of the
 * regular harmonics (themselves the degree-1 case of the addition theorem):
 *   d/dz R_n^m = R_{n-1}^m,  d/dx R_n^m = (R_{n-1}^{m+1} - R_{n-1}^{m-1}) / 2,
 *   d/dy R_n^m = -i (R_{n-1}^{m-1} + R_{n-1}^{m+1}) / 2. */
void oracle_l2p(int p, const double c[3], const double *Lin, int64_t n,
                const double *xyz, double *phi, double *grad) {
  const cplx *L = (const cplx *)Lin;
  cplx *R = malloc(sizeof(cplx) * ncoef(p));
  for (int64_t i = 0; i < n; ++i) {
    double d[3] = {xyz[3 * i] - c[0], xyz[3 * i + 1] - c[1], xyz[3 * i + 2] - c[2]};
    regular_c(p, d, R);
    cplx f = 0, gx = 0, gy = 0, gz = 0;
    for (int nn = 0; nn <= p; ++nn)
      for (int m = -nn; m <= nn; ++m) {
        cplx Lv = L[idx(nn, m)];
        f += Lv * R[idx(nn, m)];
        gx += Lv * 0.5 * (at(R, p, nn - 1, m + 1) - at(R, p, nn - 1, m - 1));
        gy += Lv * (-0.5 * I) * (at(R, p, nn - 1, m - 1) + at(R, p, nn - 1, m + 1));
        gz += Lv * at(R, p, nn - 1, m);
      }
    phi[i] += creal(f);
    if (grad) {
      grad[3 * i] += creal(gx);
      grad[3 * i + 1] += creal(gy);
      grad[3 * i + 2] += creal(gz);
    }
  }
  free(R);
}

/* M2P: phi = sum M_n^m I_n^m(x - c); derivative rules of the irregular
 * harmonics (degree-1 case of the irregular addition theorem):
 *   d/dz I_n^m = -I_{n+1}^m,  d/dx I_n^m = (I_{n+1}^{m+1} - I_{n+1}^{m-1}) / 2,
 *   d/dy I_n^m = -i (I_{n+1}^{m+1} + I_{n+1}^{m-1}) / 2. */
void oracle_m2p(int p, const double c[3], const double *Min, int64_t n,
                const double *xyz, double *phi, double *grad) {
  const cplx *M = (const cplx *)Min;
  int p1 = p + 1;
  cplx *Iv = malloc(sizeof(cplx) * ncoef(p1));
  for (int64_t i = 0; i < n; ++i) {
    double d[3] = {xyz[3 * i] - c[0], xyz[3 * i + 1] - c[1], xyz[3 * i + 2] - c[2]};
    irregular_c(p1, d, Iv);
    cplx f = 0, gx = 0, gy = 0, gz = 0;
    for (int nn = 0; nn <= p; ++nn)
      for (int m = -nn; m <= nn; ++m) {
        cplx Mv = M[idx(nn, m)];
        f += Mv * Iv[idx(nn, m)];
        gx += Mv * 0.5 * (at(Iv, p1, nn + 1, m + 1) - at(Iv, p1, nn + 1, m - 1));
        gy += Mv * (-0.5 * I) * (at(Iv, p1, nn + 1, m + 1) + at(Iv, p1, nn + 1, m - 1));
        gz -= Mv * at(Iv, p1, nn + 1, m);
      }
    phi[i] += creal(f);
    if (grad) {
      grad[3 * i] += creal(gx);
      grad[3 * i + 1] += creal(gy);
      grad[3 * i + 2] += creal(gz);
    }
  }
  free(Iv);
}

/* ------------------------------------------------------------------------
 * Root cube and Morton keys: the 3D -> 1D locality mapping of §3.1.
 * ---------------------------------------------------------------------- */
int oracle_root_cube(int64_t n, const double *xyz, double lo[3], double *D) {
  double hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = 0.0;
    hi[a] = 0.0;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double v = xyz[3 * i + a];
      if (!isfinite(v)) return -1;
      if (i == 0 || v < lo[a]) lo[a] = v;
      if (i == 0 || v > hi[a]) hi[a] = v;
    }
  double ext = 0.0;
  for (int a = 0; a < 3; ++a)
    if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
  if (ext == 0.0) {
    *D = 1.0;
  } else {
    int e;
    frexp(ext, &e); /* ext = f * 2^e, f in [0.5, 1): 2^e is the smallest power of two > ext */
    *D = ldexp(1.0, e);
  }
  return 0;
}

static uint32_t quantize(double x, double lo, double D) {
  double s = ldexp(1.0, MAXDEPTH) / D; /* power of two: the product below is exact */
  double t = floor((x - lo) * s);
  double top = (double)((1u << MAXDEPTH) - 1);
  if (t > top) t = top;
  if (t < 0) t = 0;
  return (uint32_t)t;
}

static uint64_t interleave(uint32_t qx, uint32_t qy, uint32_t qz) {
  uint64_t k = 0;
  for (int b = 0; b < MAXDEPTH; ++b) {
    k |= (uint64_t)((qx >> b) & 1u) << (3 * b);
    k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
    k |= (uint64_t)((qz >> b) & 1u) << (3 * b + 2);
  }
  return k;
}

static void deinterleave(uint64_t k, int nbits, int32_t a[3]) {
  a[0] = a[1] = a[2] = 0;
  for (int b = 0; b < nbits; ++b) {
    a[0] |= (int32_t)((k >> (3 * b)) & 1u) << b;
    a[1] |= (int32_t)((k >> (3 * b + 1)) & 1u) << b;
    a[2] |= (int32_t)((k >> (3 * b + 2)) & 1u) << b;
  }
}

void oracle_morton_keys(int64_t n, const double *xyz, const double lo[3], double D,
                        uint64_t *keys) {
  for (int64_t i = 0; i < n; ++i)
    keys[i] = interleave(quantize(xyz[3 * i], lo[0], D), quantize(xyz[3 * i + 1], lo[1], D),
                         quantize(xyz[3 * i + 2], lo[2], D));
}

/* ------------------------------------------------------------------------
 * Tree and lists (§2.2 interaction list; adaptive U/W/X lists).
 * ---------------------------------------------------------------------- */
static void ivec_push(ivec *v, int32_t x) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 16;
    v->a = realloc(v->a, sizeof(int32_t) * v->cap);
  }
  v->a[v->n++] = x;
}


typedef struct {
  uint64_t key;
  int32_t i;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
  const keyidx *x = a, *y = b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->i < y->i ? -1 : (x->i > y->i);
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y);
}

/* two boxes are adjacent iff their closed cubes, mapped to the finest integer
 * grid, intersect on every axis (a box is adjacent to itself) */
static int adjacent(const oracle_tree *t, int32_t A, int32_t B) {
  int sa = MAXDEPTH - t->box_level[A], sb = MAXDEPTH - t->box_level[B];
  for (int a = 0; a < 3; ++a) {
    int64_t alo = (int64_t)t->anchor[A][a] << sa, ahi = ((int64_t)t->anchor[A][a] + 1) << sa;
    int64_t blo = (int64_t)t->anchor[B][a] << sb, bhi = ((int64_t)t->anchor[B][a] + 1) << sb;
    if (alo > bhi || blo > ahi) return 0;
  }
  return 1;
}

/* U(B): leaves adjacent to B; W(B): boxes deeper than B, not adjacent to B,
 * whose parent is adjacent to B.  Every ancestor of a box adjacent to B is
 * adjacent to B, so a descent through adjacent boxes from the root finds
 * both. */
static void descend_uw(oracle_tree *t, int32_t B, int32_t Q) {
  if (adjacent(t, Q, B)) {
    if (t->box_nchild[Q] == 0) {
      ivec_push(&t->U[B], Q);
    } else {
      for (int c = 0; c < t->box_nchild[Q]; ++c) descend_uw(t, B, t->box_child[Q] + c);
    }
  } else if (t->box_level[Q] > t->box_level[B]) {
    ivec_push(&t->W[B], Q); /* reached only through an adjacent parent */
  }
}

oracle_tree *oracle_tree_build(int64_t n, const double *xyz, int leaf_size, int max_depth) {
  if (n < 0 || leaf_size < 1 || max_depth < 0 || max_depth > MAXDEPTH) return NULL;
  oracle_tree *t = calloc(1, sizeof(oracle_tree));
  t->n = n;
  t->leaf_size = leaf_size;
  t->max_depth = max_depth;
  if (oracle_root_cube(n, xyz, t->lo, &t->D) != 0) {
    free(t);
    return NULL;
  }
  uint64_t *raw = malloc(sizeof(uint64_t) * (n ? n : 1));
  oracle_morton_keys(n, xyz, t->lo, t->D, raw);
  keyidx *ki = malloc(sizeof(keyidx) * (n ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    ki[i].key = raw[i];
    ki[i].i = (int32_t)i;
  }
  /* ordering by (key, input index) = a stable sort by key */
  qsort(ki, n, sizeof(keyidx), cmp_keyidx);
  t->keys = malloc(sizeof(uint64_t) * (n ? n : 1));
  t->perm = malloc(sizeof(int32_t) * (n ? n : 1));
  t->xyz = malloc(sizeof(double) * 3 * (n ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    t->keys[i] = ki[i].key;
    t->perm[i] = ki[i].i;
    for (int a = 0; a < 3; ++a) t->xyz[3 * i + a] = xyz[3 * (int64_t)ki[i].i + a];
  }
  free(ki);
  free(raw);

  /* boxes, level by level; children of one box are consecutive and boxes of
   * a level are in key order, so the index order is (level, key) */
  int64_t cap = 1024, nb = 0;
  t->box_key = malloc(sizeof(uint64_t) * cap);
  t->box_level = malloc(sizeof(int32_t) * cap);
  t->box_first = malloc(sizeof(int32_t) * cap);
  t->box_count = malloc(sizeof(int32_t) * cap);
  t->box_parent = malloc(sizeof(int32_t) * cap);
  t->level_offset = malloc(sizeof(int32_t) * (MAXDEPTH + 2));
  t->nlevels = 0;
  t->level_offset[0] = 0;
  if (n > 0) {
    t->box_key[0] = 0;
    t->box_level[0] = 0;
    t->box_first[0] = 0;
    t->box_count[0] = (int32_t)n;
    t->box_parent[0] = -1;
    nb = 1;
    t->nlevels = 1;
    t->level_offset[1] = 1;
    for (int l = 0; l < max_depth; ++l) {
      int64_t b0 = t->level_offset[l], b1 = t->level_offset[l + 1];
      int shift = 3 * (MAXDEPTH - (l + 1));
      for (int64_t b = b0; b < b1; ++b) {
        if (t->box_count[b] <= leaf_size) continue;
        int64_t f = t->box_first[b], e = f + t->box_count[b];
        for (int64_t i = f; i < e;) {
          uint64_t pre = t->keys[i] >> shift;
          int64_t j = i;
          while (j < e && (t->keys[j] >> shift) == pre) ++j;
          if (nb == cap) {
            cap *= 2;
            t->box_key = realloc(t->box_key, sizeof(uint64_t) * cap);
            t->box_level = realloc(t->box_level, sizeof(int32_t) * cap);
            t->box_first = realloc(t->box_first, sizeof(int32_t) * cap);
            t->box_count = realloc(t->box_count, sizeof(int32_t) * cap);
            t->box_parent = realloc(t->box_parent, sizeof(int32_t) * cap);
          }
          t->box_key[nb] = pre;
          t->box_level[nb] = l + 1;
          t->box_first[nb] = (int32_t)i;
          t->box_count[nb] = (int32_t)(j - i);
          t->box_parent[nb] = (int32_t)b;
          ++nb;
          i = j;
        }
      }
      if (nb == b1) break;
      t->nlevels = l + 2;
      t->level_offset[l + 2] = (int32_t)nb;
    }
  }
  t->nboxes = nb;
  int64_t nba = nb ? nb : 1;
  t->box_child = malloc(sizeof(int32_t) * nba);
  t->box_nchild = calloc(nba, sizeof(int32_t));
  t->anchor = malloc(sizeof(int32_t[3]) * nba);
  t->center = malloc(sizeof(double[3]) * nba);
  t->side = malloc(sizeof(double) * (MAXDEPTH + 1));
  for (int l = 0; l <= MAXDEPTH; ++l) t->side[l] = ldexp(t->D, -l);
  for (int64_t b = 0; b < nb; ++b) t->box_child[b] = -1;
  for (int64_t b = 1; b < nb; ++b) {
    int32_t P = t->box_parent[b];
    if (t->box_nchild[P] == 0) t->box_child[P] = (int32_t)b;
    t->box_nchild[P]++;
  }
  for (int64_t b = 0; b < nb; ++b) {
    deinterleave(t->box_key[b], t->box_level[b], t->anchor[b]);
    double a = t->side[t->box_level[b]];
    for (int k = 0; k < 3; ++k) t->center[b][k] = t->lo[k] + ((double)t->anchor[b][k] + 0.5) * a;
  }

  /* colleagues: same-level adjacent boxes other than B; they are children of
   * parent(B) or of its colleagues (§2.2 "parent's neighbours' children") */
  ivec *col = calloc(nba, sizeof(ivec));
  for (int64_t b = 1; b < nb; ++b) {
    int32_t P = t->box_parent[b];
    ivec cand = {0};
    ivec_push(&cand, P);
    for (int64_t k = 0; k < col[P].n; ++k) ivec_push(&cand, col[P].a[k]);
    for (int64_t k = 0; k < cand.n; ++k) {
      int32_t C = cand.a[k];
      for (int c = 0; c < t->box_nchild[C]; ++c) {
        int32_t A = t->box_child[C] + c;
        if (A != b && adjacent(t, A, (int32_t)b)) ivec_push(&col[b], A);
      }
    }
    free(cand.a);
    qsort(col[b].a, col[b].n, sizeof(int32_t), cmp_i32);
  }

  t->U = calloc(nba, sizeof(ivec));
  t->V = calloc(nba, sizeof(ivec));
  t->W = calloc(nba, sizeof(ivec));
  t->X = calloc(nba, sizeof(ivec));
  /* V(B), level >= 2: children of the colleagues of parent(B) that are not
   * adjacent to B (at most 6^3 - 3^3 = 189) */
  for (int64_t b = 1; b < nb; ++b) {
    if (t->box_level[b] < 2) continue;
    int32_t P = t->box_parent[b];
    for (int64_t k = 0; k < col[P].n; ++k) {
      int32_t C = col[P].a[k];
      for (int c = 0; c < t->box_nchild[C]; ++c) {
        int32_t A = t->box_child[C] + c;
        if (!adjacent(t, A, (int32_t)b)) ivec_push(&t->V[b], A);
      }
    }
    qsort(t->V[b].a, t->V[b].n, sizeof(int32_t), cmp_i32);
  }
  /* U and W of every leaf */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t b = 0; b < nb; ++b) {
    if (t->box_nchild[b] != 0) continue;
    descend_uw(t, (int32_t)b, 0);
    qsort(t->U[b].a, t->U[b].n, sizeof(int32_t), cmp_i32);
    qsort(t->W[b].a, t->W[b].n, sizeof(int32_t), cmp_i32);
  }
  /* X(C) = { leaf A : C in W(A) } */
  for (int64_t b = 0; b < nb; ++b)
    for (int64_t k = 0; k < t->W[b].n; ++k) ivec_push(&t->X[t->W[b].a[k]], (int32_t)b);
  for (int64_t b = 0; b < nb; ++b) qsort(t->X[b].a, t->X[b].n, sizeof(int32_t), cmp_i32);

  for (int64_t b = 0; b < nb; ++b) free(col[b].a);
  free(col);
  return t;
}

/* Direct evaluation of small well-separated leaf pairs (the adaptive FMM's
 * practice for W/X interactions whose boxes hold few points): a pair of leaves
 * (B, A) with A in W(B) and A holding at most max_points points moves, in both
 * directions, to the near field -- A joins U(B) and B joins U(A), A leaves
 * W(B) and B leaves X(A) -- so B's targets see A's points by the direct sum
 * instead of M2P, and A's targets see B's points by the direct sum instead of
 * P2L + L2P.  The operator stays symmetric.  Rows stay sorted. */
void oracle_tree_direct_wx(oracle_tree *t, int max_points) {
  if (!t || max_points < 1) return;
  for (int64_t b = 0; b < t->nboxes; ++b) {
    if (t->box_nchild[b] != 0) continue;
    ivec keep = {0};
    for (int64_t k = 0; k < t->W[b].n; ++k) {
      int32_t A = t->W[b].a[k];
      if (t->box_nchild[A] == 0 && t->box_count[A] <= max_points) {
        ivec_push(&t->U[b], A);
        ivec_push(&t->U[A], (int32_t)b);
        /* remove b from X(A) */
        ivec *x = &t->X[A];
        int64_t w = 0;
        for (int64_t i = 0; i < x->n; ++i)
          if (x->a[i] != (int32_t)b) x->a[w++] = x->a[i];
        x->n = w;
      } else {
        ivec_push(&keep, A);
      }
    }
    free(t->W[b].a);
    t->W[b] = keep;
  }
  for (int64_t b = 0; b < t->nboxes; ++b)
    if (t->box_nchild[b] == 0) qsort(t->U[b].a, t->U[b].n, sizeof(int32_t), cmp_i32);
}

void oracle_tree_free(oracle_tree *t) {
  if (!t) return;
  int64_t nba = t->nboxes ? t->nboxes : 1;
  for (int64_t b = 0; b < t->nboxes; ++b) {
    free(t->U[b].a);
    free(t->V[b].a);
    free(t->W[b].a);
    free(t->X[b].a);
  }
  (void)nba;
  free(t->U);
  free(t->V);
  free(t->W);
  free(t->X);
  free(t->keys);
  free(t->perm);
  free(t->xyz);
  free(t->level_offset);
  free(t->box_key);
  free(t->box_level);
  free(t->box_first);
  free(t->box_count);
  free(t->box_parent);
  free(t->box_child);
  free(t->box_nchild);
  free(t->anchor);
  free(t->center);
  free(t->side);
  free(t);
}

static int64_t list_total(const ivec *L, int64_t nb) {
  int64_t s = 0;
  for (int64_t b = 0; b < nb; ++b) s += L[b].n;
  return s;
}

void oracle_tree_sizes(const oracle_tree *t, int64_t s[7]) {
  s[0] = t->n;
  s[1] = t->nboxes;
  s[2] = t->nlevels;
  s[3] = list_total(t->U, t->nboxes);
  s[4] = list_total(t->V, t->nboxes);
  s[5] = list_total(t->W, t->nboxes);
  s[6] = list_total(t->X, t->nboxes);
}

void oracle_tree_geometry(const oracle_tree *t, double lo[3], double *D) {
  for (int a = 0; a < 3; ++a) lo[a] = t->lo[a];
  *D = t->D;
}

static void export_list(const ivec *L, int64_t nb, int32_t *off, int32_t *ix) {
  int64_t s = 0;
  for (int64_t b = 0; b < nb; ++b) {
    if (off) off[b] = (int32_t)s;
    if (ix) memcpy(ix + s, L[b].a, sizeof(int32_t) * L[b].n);
    s += L[b].n;
  }
  if (off) off[nb] = (int32_t)s;
}

void oracle_tree_export(const oracle_tree *t, uint64_t *keys, int32_t *perm,
                        int32_t *level_offset, uint64_t *box_key, int32_t *box_level,
                        int32_t *box_first, int32_t *box_count, int32_t *box_parent,
                        int32_t *box_child, int32_t *box_nchild, int32_t *u_off,
                        int32_t *u_idx, int32_t *v_off, int32_t *v_idx, int32_t *w_off,
                        int32_t *w_idx, int32_t *x_off, int32_t *x_idx) {
  int64_t n = t->n, nb = t->nboxes;
  if (keys) memcpy(keys, t->keys, sizeof(uint64_t) * n);
  if (perm) memcpy(perm, t->perm, sizeof(int32_t) * n);
  if (level_offset) memcpy(level_offset, t->level_offset, sizeof(int32_t) * (t->nlevels + 1));
  if (box_key) memcpy(box_key, t->box_key, sizeof(uint64_t) * nb);
  if (box_level) memcpy(box_level, t->box_level, sizeof(int32_t) * nb);
  if (box_first) memcpy(box_first, t->box_first, sizeof(int32_t) * nb);
  if (box_count) memcpy(box_count, t->box_count, sizeof(int32_t) * nb);
  if (box_parent) memcpy(box_parent, t->box_parent, sizeof(int32_t) * nb);
  if (box_child) memcpy(box_child, t->box_child, sizeof(int32_t) * nb);
  if (box_nchild) memcpy(box_nchild, t->box_nchild, sizeof(int32_t) * nb);
  export_list(t->U, nb, u_off, u_idx);
  export_list(t->V, nb, v_off, v_idx);
  export_list(t->W, nb, w_off, w_idx);
  export_list(t->X, nb, x_off, x_idx);
}

/* ------------------------------------------------------------------------
 * FMM mat-vec (§1: analytic FMM = matrix-free H^2 mat-vec).  Pass order:
 * P2M at leaves; M2M up to level 1; at every level >= 2, M2L over V and P2L
 * over X; L2L down; at leaf targets L2P + M2P over W + P2P over U.
 * ---------------------------------------------------------------------- */
void oracle_fmm_eval(const oracle_tree *t, int p, const double *q_in, double *phi_out,
                     double *grad_out) {
  int64_t n = t->n, nb = t->nboxes;
  int nc = ncoef(p);
  if (n == 0) return;
  double *q = malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; ++i) q[i] = q_in[t->perm[i]];
  cplx *M = calloc((size_t)nb * nc, sizeof(cplx));
  cplx *L = calloc((size_t)nb * nc, sizeof(cplx));
  double *phi = calloc(n, sizeof(double));
  double *grad = calloc(3 * n, sizeof(double));

  /* P2M at every leaf */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nb; ++b)
    if (t->box_nchild[b] == 0)
      oracle_p2m(p, t->center[b], t->box_count[b], t->xyz + 3 * (int64_t)t->box_first[b],
                 q + t->box_first[b], (double *)(M + (size_t)b * nc));
  /* M2M, deepest parents first: each parent gathers its children */
  for (int l = t->nlevels - 2; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = t->level_offset[l]; b < t->level_offset[l + 1]; ++b)
      for (int c = 0; c < t->box_nchild[b]; ++c) {
        int32_t C = t->box_child[b] + c;
        oracle_m2m(p, t->center[C], (double *)(M + (size_t)C * nc), t->center[b],
                   (double *)(M + (size_t)b * nc));
      }
  }
  /* far field at every box of level >= 2: M2L over V, P2L over X */
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nb; ++b) {
    if (t->box_level[b] < 2) continue;
    for (int64_t k = 0; k < t->V[b].n; ++k) {
      int32_t A = t->V[b].a[k];
      oracle_m2l(p, t->center[A], (double *)(M + (size_t)A * nc), t->center[b],
                 (double *)(L + (size_t)b * nc));
    }
    for (int64_t k = 0; k < t->X[b].n; ++k) {
      int32_t A = t->X[b].a[k];
      oracle_p2l(p, t->center[b], t->box_count[A], t->xyz + 3 * (int64_t)t->box_first[A],
                 q + t->box_first[A], (double *)(L + (size_t)b * nc));
    }
  }
  /* L2L from level 2 down: each child gathers from its parent */
  for (int l = 3; l < t->nlevels; ++l) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = t->level_offset[l]; b < t->level_offset[l + 1]; ++b) {
      int32_t P = t->box_parent[b];
      oracle_l2l(p, t->center[P], (double *)(L + (size_t)P * nc), t->center[b],
                 (double *)(L + (size_t)b * nc));
    }
  }
  /* evaluation at the targets of every leaf */
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < nb; ++b) {
    if (t->box_nchild[b] != 0) continue;
    int64_t f = t->box_first[b], cnt = t->box_count[b];
    const double *tx = t->xyz + 3 * f;
    oracle_l2p(p, t->center[b], (double *)(L + (size_t)b * nc), cnt, tx, phi + f, grad + 3 * f);
    for (int64_t k = 0; k < t->W[b].n; ++k) {
      int32_t A = t->W[b].a[k];
      oracle_m2p(p, t->center[A], (double *)(M + (size_t)A * nc), cnt, tx, phi + f, grad + 3 * f);
    }
    for (int64_t k = 0; k < t->U[b].n; ++k) {
      int32_t A = t->U[b].a[k];
      int64_t fa = t->box_first[A], ca = t->box_count[A];
      for (int64_t i = 0; i < cnt; ++i)
        for (int64_t j = fa; j < fa + ca; ++j) {
          double dx = tx[3 * i] - t->xyz[3 * j];
          double dy = tx[3 * i + 1] - t->xyz[3 * j + 1];
          double dz = tx[3 * i + 2] - t->xyz[3 * j + 2];
          double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 == 0.0) continue;
          double r = sqrt(r2);
          phi[f + i] += q[j] / r;
          double s = q[j] / (r2 * r);
          grad[3 * (f + i)] -= s * dx;
          grad[3 * (f + i) + 1] -= s * dy;
          grad[3 * (f + i) + 2] -= s * dz;
        }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    int32_t o = t->perm[i];
    phi_out[o] = phi[i];
    if (grad_out)
      for (int a = 0; a < 3; ++a) grad_out[3 * (int64_t)o + a] = grad[3 * i + a];
  }
  free(q);
  free(M);
  free(L);
  free(phi);
  free(grad);
}

/* ------------------------------------------------------------------------
 * Dual-tree traversal with a multipole acceptance criterion (§2.1: Dehnen's
 * dual tree walk as the alternative to fixed interaction lists).
 *
 * Expansion centres are the geometric box centres.  Cell radius:
 *   r_B = max over the points j of B of |x_j - c_B|.
 * A pair (T, S) of distinct cells is accepted for one M2L from S into T iff
 *   r_T + r_S < theta |c_T - c_S|,
 * with c_T - c_S taken from the integer anchors (exact in FP64) and every
 * operation a single IEEE-rounded add, multiply or square root in the order
 * written, so that another implementation that follows the same steps takes
 * the same decisions.
 * A rejected pair splits by a rule that does not depend on the order of T
 * and S, so (T, S) ends in M2L (or P2P) exactly when (S, T) does and the
 * truncated operator stays symmetric:
 *   both leaves       -> P2P (T == S included: the leaf with itself)
 *   one leaf          -> split the other cell
 *   different levels  -> split the coarser cell
 *   same level        -> split both.
 * Starting from (root, root) every ordered pair (target point, source point)
 * lands in exactly one M2L pair (T, S) with the target in T and the source in
 * S, or in one P2P pair of leaves.
 * ---------------------------------------------------------------------- */
struct oracle_dual {
  int64_t nb;
  double theta;
  double *radius;
  ivec *M, *P; /* per target box: M2L sources, P2P source leaves */
};

static int dual_accept(const oracle_tree *t, const double *r, double theta, int32_t T,
                       int32_t S) {
  double aT = t->side[t->box_level[T]], aS = t->side[t->box_level[S]];
  double d[3];
  for (int k = 0; k < 3; ++k)
    d[k] = ((double)t->anchor[T][k] + 0.5) * aT - ((double)t->anchor[S][k] + 0.5) * aS;
  double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  return r[T] + r[S] < theta * dist;
}

static void dual_walk(const oracle_tree *t, oracle_dual *D, int32_t T, int32_t S) {
  if (T != S && dual_accept(t, D->radius, D->theta, T, S)) {
    ivec_push(&D->M[T], S);
    return;
  }
  int lt = t->box_nchild[T] == 0, ls = t->box_nchild[S] == 0;
  if (lt && ls) {
    ivec_push(&D->P[T], S);
    return;
  }
  int splitT, splitS;
  if (lt) {
    splitT = 0;
    splitS = 1;
  } else if (ls) {
    splitT = 1;
    splitS = 0;
  } else if (t->box_level[T] != t->box_level[S]) {
    splitT = t->box_level[T] < t->box_level[S];
    splitS = !splitT;
  } else {
    splitT = splitS = 1;
  }
  int nt = splitT ? t->box_nchild[T] : 1, ns = splitS ? t->box_nchild[S] : 1;
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < ns; ++j)
      dual_walk(t, D, splitT ? t->box_child[T] + i : T, splitS ? t->box_child[S] + j : S);
}

oracle_dual *oracle_dual_build(const oracle_tree *t, double theta) {
  oracle_dual *D = calloc(1, sizeof(oracle_dual));
  int64_t nb = t->nboxes, nba = nb ? nb : 1;
  D->nb = nb;
  D->theta = theta;
  D->radius = calloc(nba, sizeof(double));
  D->M = calloc(nba, sizeof(ivec));
  D->P = calloc(nba, sizeof(ivec));
  for (int64_t b = 0; b < nb; ++b) {
    double m = 0.0;
    for (int64_t j = t->box_first[b]; j < t->box_first[b] + t->box_count[b]; ++j) {
      double dx = t->xyz[3 * j] - t->center[b][0];
      double dy = t->xyz[3 * j + 1] - t->center[b][1];
      double dz = t->xyz[3 * j + 2] - t->center[b][2];
      double s = dx * dx + dy * dy + dz * dz;
      if (s > m) m = s;
    }
    D->radius[b] = sqrt(m);
  }
  if (nb > 0) dual_walk(t, D, 0, 0);
  for (int64_t b = 0; b < nb; ++b) {
    qsort(D->M[b].a, D->M[b].n, sizeof(int32_t), cmp_i32);
    qsort(D->P[b].a, D->P[b].n, sizeof(int32_t), cmp_i32);
  }
  return D;
}

void oracle_dual_free(oracle_dual *D) {
  if (!D) return;
  for (int64_t b = 0; b < D->nb; ++b) {
    free(D->M[b].a);
    free(D->P[b].a);
  }
  free(D->M);
  free(D->P);
  free(D->radius);
  free(D);
}

void oracle_dual_sizes(const oracle_dual *D, int64_t s[2]) {
  s[0] = list_total(D->M, D->nb);
  s[1] = list_total(D->P, D->nb);
}

void oracle_dual_export(const oracle_dual *D, int32_t *m_off, int32_t *m_idx, int32_t *p_off,
                        int32_t *p_idx, double *radius) {
  export_list(D->M, D->nb, m_off, m_idx);
  export_list(D->P, D->nb, p_off, p_idx);
  if (radius) memcpy(radius, D->radius, sizeof(double) * D->nb);
}

/* FMM mat-vec on the dual-tree lists: P2M at leaves; M2M up to the root;
 * M2L over every accepted pair (any level, cells of different sizes
 * included); L2L from the root down; at leaf targets L2P + P2P over the
 * leaf pairs.  There are no W/X corrections: the traversal covers every
 * point pair by M2L or P2P. */
void oracle_dual_eval(const oracle_tree *t, const oracle_dual *D, int p, const double *q_in,
                      double *phi_out, double *grad_out) {
  int64_t n = t->n, nb = t->nboxes;
  int nc = ncoef(p);
  if (n == 0) return;
  double *q = malloc(sizeof(double) * n);
  for (int64_t i = 0; i < n; ++i) q[i] = q_in[t->perm[i]];
  cplx *M = calloc((size_t)nb * nc, sizeof(cplx));
  cplx *L = calloc((size_t)nb * nc, sizeof(cplx));
  double *phi = calloc(n, sizeof(double));
  double *grad = calloc(3 * n, sizeof(double));

#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nb; ++b)
    if (t->box_nchild[b] == 0)
      oracle_p2m(p, t->center[b], t->box_count[b], t->xyz + 3 * (int64_t)t->box_first[b],
                 q + t->box_first[b], (double *)(M + (size_t)b * nc));
  for (int l = t->nlevels - 2; l >= 0; --l) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = t->level_offset[l]; b < t->level_offset[l + 1]; ++b)
      for (int c = 0; c < t->box_nchild[b]; ++c) {
        int32_t C = t->box_child[b] + c;
        oracle_m2m(p, t->center[C], (double *)(M + (size_t)C * nc), t->center[b],
                   (double *)(M + (size_t)b * nc));
      }
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nb; ++b)
    for (int64_t k = 0; k < D->M[b].n; ++k) {
      int32_t A = D->M[b].a[k];
      oracle_m2l(p, t->center[A], (double *)(M + (size_t)A * nc), t->center[b],
                 (double *)(L + (size_t)b * nc));
    }
  for (int l = 1; l < t->nlevels; ++l) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = t->level_offset[l]; b < t->level_offset[l + 1]; ++b) {
      int32_t P = t->box_parent[b];
      oracle_l2l(p, t->center[P], (double *)(L + (size_t)P * nc), t->center[b],
                 (double *)(L + (size_t)b * nc));
    }
  }
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t b = 0; b < nb; ++b) {
    if (t->box_nchild[b] != 0) continue;
    int64_t f = t->box_first[b], cnt = t->box_count[b];
    const double *tx = t->xyz + 3 * f;
    oracle_l2p(p, t->center[b], (double *)(L + (size_t)b * nc), cnt, tx, phi + f, grad + 3 * f);
    for (int64_t k = 0; k < D->P[b].n; ++k) {
      int32_t A = D->P[b].a[k];
      int64_t fa = t->box_first[A], ca = t->box_count[A];
      for (int64_t i = 0; i < cnt; ++i)
        for (int64_t j = fa; j < fa + ca; ++j) {
          double dx = tx[3 * i] - t->xyz[3 * j];
          double dy = tx[3 * i + 1] - t->xyz[3 * j + 1];
          double dz = tx[3 * i + 2] - t->xyz[3 * j + 2];
          double r2 = dx * dx + dy * dy + dz * dz;
          if (r2 == 0.0) continue;
          double r = sqrt(r2);
          phi[f + i] += q[j] / r;
          double s = q[j] / (r2 * r);
          grad[3 * (f + i)] -= s * dx;
          grad[3 * (f + i) + 1] -= s * dy;
          grad[3 * (f + i) + 2] -= s * dz;
        }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    int32_t o = t->perm[i];
    phi_out[o] = phi[i];
    if (grad_out)
      for (int a = 0; a < 3; ++a) grad_out[3 * (int64_t)o + a] = grad[3 * i + a];
  }
  free(q);
  free(M);
  free(L);
  free(phi);
  free(grad);
}

// helmholtz.cu -- FMM mat-vec with the Helmholtz kernel e^{i kappa r}/r (the
// paper's second kernel: §1 sets FMM against HSS for Laplace and Helmholtz
// kernels, §4.2 preconditions the Helmholtz equation with kappa = 7 on
// [-1, 1]^3), FP64 complex, on a plan's octree and U/V/W/X lists.
//
// Expansions (low-frequency form of Gegenbauer's addition theorem; the paper
// prints none):
//   Y_n^m   orthonormal spherical harmonics, Condon-Shortley phase,
//           Y_n^{-m} = (-1)^m conj(Y_n^m);
//   R_n^m(x) = j_n(kappa|x|) Y_n^m(x^),  S_n^m(x) = h_n(kappa|x|) Y_n^m(x^),
//           h_n = j_n + i y_n;
//   multipole  phi(x) = sum M_n^m S_n^m(x - c),  P2M: M += 4 pi i kappa q conj(R(y - c));
//   local      phi(x) = sum L_n^m R_n^m(x - c),  P2L: L += 4 pi i kappa q h_n conj(Y((y - c)^));
//   translations T(t)_{(n'm'),(nm)} = 4 pi sum_l i^{n'+l-n} X_l^{m-m'}(t) G(n,m; n',m'; l)
//           with the Gaunt coefficients G = int Y_n^m conj(Y_n'^m') conj(Y_l^{m-m'}):
//           X = S for M2L (t = c_target - c_source), X = R for M2M (t = c_parent -
//           c_child) and L2L (t = c_child - c_parent).
// Unlike the Laplace operators these are not scale-free: kappa times the box
// side changes from level to level, so every level has its own 316 M2L and
// 8 + 8 M2M / L2L matrices.  They are assembled on the device from a Gaunt
// table and per-operator tables of X_l^mu(t), both computed on the host.
//
// Passes: q to sorted order; P2M (leaves); M2M (levels upwards); M2L (V) and
// P2L (X) at levels >= 2; L2L (levels downwards); L2P + M2P (W) per leaf;
// P2P (U) per leaf, which adds the far field and stores phi at the input
// index.  Every pass is a plain CUDA-core kernel in FP64: GB300's FP64 rate is
// the bound (4 FP64 FMAs per complex multiply-add in the translations; a
// square root, a division and a sine/cosine pair per near-field pair).  A
// plan of mixed precision runs M2L (with per-level scalings) and the near
// field in FP32 (the low-accuracy use of §4.2); P2M, M2M, L2L, P2L, L2P and
// M2P stay FP64.
#include <cmath>
#include <complex>
#include <mutex>
#include <vector>

#include "plan.cuh"

namespace fmm {

namespace {

constexpr int kHelmMaxOrder = 12;
constexpr int kHelmMaxNC = (kHelmMaxOrder + 1) * (kHelmMaxOrder + 1);
constexpr int kHelmBatch = 32;  // points staged per P2M / P2L batch
constexpr int kHelmThreads = 128;
constexpr double kPi = 3.141592653589793238462643383279502884;

// recurrence constants of the normalised harmonics (filled once per process):
//   sectoral  Y_m^m = c_sec[m] * w * Y_{m-1}^{m-1},  w = (x + iy)/r,
//             c_sec[m] = -sqrt((2m+1)/(2m));
//   first     Y_{m+1}^m = sqrt(2m+3) u Y_m^m,  u = z/r;
//   column    Y_n^m = c_a[n,m] (u Y_{n-1}^m - c_b[n,m] Y_{n-2}^m),
//             c_a = sqrt((4n^2-1)/(n^2-m^2)), c_b = sqrt(((n-1)^2-m^2)/(4(n-1)^2-1)).
__constant__ double c_sec[kHelmMaxOrder + 1];
__constant__ double c_first[kHelmMaxOrder + 1];
__constant__ double c_a[kHelmMaxNC];
__constant__ double c_b[kHelmMaxNC];

__host__ __device__ constexpr int hc(int n, int m) { return n * n + n + m; }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a b
__device__ __forceinline__ double2 cmad(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Spherical Bessel functions j_0..j_p (and y_0..y_p when WANT_Y) at x >= 0.
//  x < 1: the power series of j_n (terms fall monotonically);
//  x >= 1: downward (Miller) recurrence f_{n-1} = (2n+1)/x f_n - f_{n+1} from
//          (f_{N+1}, f_N) = (0, 1), N = p + x + 32, normalised by whichever of
//          j_0 = sin x / x, j_1 = sin x / x^2 - cos x / x is larger;
//  y_n: upward recurrence from y_0 = -cos x / x, y_1 = -cos x / x^2 - sin x / x.
__host__ __device__ __forceinline__ void sin_cos(double x, double *s, double *c) {
#ifdef __CUDA_ARCH__
  sincos(x, s, c);
#else
  *s = std::sin(x);
  *c = std::cos(x);
#endif
}

template <bool WANT_Y>
__host__ __device__ void sph_bessel(int p, double x, double *j, double *y) {
  if (x < 1.0) {
    double lead = 1.0;
    const double h = -0.5 * x * x;
    for (int n = 0; n <= p; ++n) {
      if (n > 0) lead *= x / (2.0 * n + 1.0);
      double sum = 1.0, term = 1.0;
      for (int k = 1; k < 40; ++k) {
        term *= h / ((double)k * (2.0 * n + 2.0 * k + 1.0));
        sum += term;
        if (fabs(term) < 1e-17 * fabs(sum)) break;
      }
      j[n] = lead * sum;
    }
  } else {
    const double ix = 1.0 / x;
    const int N = p + (int)x + 32;
    double f1 = 0.0, f0 = 1.0;  // f_{n+1}, f_n
    for (int n = N; n > p; --n) {
      const double fm = (2.0 * n + 1.0) * ix * f0 - f1;
      f1 = f0;
      f0 = fm;
      if (fabs(f0) > 1e200) {
        f0 *= 1e-200;
        f1 *= 1e-200;
      }
    }
    j[p] = f0;
    for (int n = p; n >= 1; --n) {
      const double fm = (2.0 * n + 1.0) * ix * f0 - f1;
      f1 = f0;
      f0 = fm;
      j[n - 1] = f0;
      if (fabs(f0) > 1e200) {
        for (int k = n - 1; k <= p; ++k) j[k] *= 1e-200;
        f0 *= 1e-200;
        f1 *= 1e-200;
      }
    }
    double s, c;
    sin_cos(x, &s, &c);
    const double j0 = s * ix, j1 = (s * ix - c) * ix;
    const double scale = fabs(j0) >= fabs(j1) ? j0 / j[0] : j1 / (p >= 1 ? j[1] : f1);
    for (int n = 0; n <= p; ++n) j[n] *= scale;
  }
  if (WANT_Y) {
    const double ix = 1.0 / x;
    double s, c;
    sin_cos(x, &s, &c);
    y[0] = -c * ix;
    if (p >= 1) y[1] = (-c * ix - s) * ix;
    for (int n = 1; n < p; ++n) y[n + 1] = (2.0 * n + 1.0) * ix * y[n] - y[n - 1];
  }
}

// Calls f(n, m, Y_n^m) for 0 <= m <= n <= p, m outer, n inner, for the
// direction of d (the +z axis when d = 0).
template <typename F>
__device__ __forceinline__ void for_harmonics(int p, double dx, double dy, double dz, F &&f) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  double u = 1.0;
  double2 w = make_double2(0.0, 0.0);
  if (r2 > 0.0) {
    const double ir = rsqrt(r2);
    u = dz * ir;
    w = make_double2(dx * ir, dy * ir);
  }
  double2 ymm = make_double2(0.28209479177387814347403972578038629, 0.0);  // 1/sqrt(4 pi)
  for (int m = 0; m <= p; ++m) {
    if (m > 0) ymm = cscale(cmul(w, ymm), c_sec[m]);
    f(m, m, ymm);
    if (m == p) break;
    double2 y2 = ymm;
    double2 y1 = cscale(ymm, c_first[m] * u);
    f(m + 1, m, y1);
    for (int n = m + 2; n <= p; ++n) {
      const int i = hc(n, m);
      const double2 y0 = cscale(make_double2(fma(u, y1.x, -c_b[i] * y2.x), fma(u, y1.y, -c_b[i] * y2.y)),
                                c_a[i]);
      f(n, m, y0);
      y2 = y1;
      y1 = y0;
    }
  }
}

// ---------------------------------------------------------------- operators
// op[o][k][j] = 4 pi sum_l i^{n_j + l - n_k} X[o][l, m_k - m_j] G(k; j; l): one
// thread per (operator, input k, output j); input-major so that the threads
// of a translation (one per output j) read consecutive addresses.
__global__ void k_h_assemble(int64_t nops, int p, const double2 *__restrict__ X,
                             const double *__restrict__ gaunt, double2 *__restrict__ op) {
  const int NC = (p + 1) * (p + 1), NX = (2 * p + 1) * (2 * p + 1);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nops * NC * NC) return;
  const int64_t o = e / ((int64_t)NC * NC);
  const int kj = (int)(e - o * NC * NC), k = kj / NC, jj = kj % NC;
  const int n = (int)sqrtf((float)k + 0.5f), m = k - n * n - n;
  const int n2 = (int)sqrtf((float)jj + 0.5f), m2 = jj - n2 * n2 - n2;
  const int mu = m - m2, l0 = abs(n - n2);
  const double *g = gaunt + ((int64_t)k * NC + jj) * (p + 1);
  const double2 *x = X + o * NX;
  double2 acc = make_double2(0.0, 0.0);
  for (int l = l0; l <= n + n2; l += 2) {
    if (abs(mu) > l) continue;
    const double s = (((n2 + l - n) >> 1) & 1) ? -g[(l - l0) >> 1] : g[(l - l0) >> 1];
    const double2 v = x[hc(l, mu)];
    acc.x = fma(s, v.x, acc.x);
    acc.y = fma(s, v.y, acc.y);
  }
  op[e] = cscale(acc, 4.0 * kPi);
}

// ---------------------------------------------------------------- passes
struct HGeo {
  double lo[3];
  double kappa;
};

__device__ __forceinline__ void box_center(const BoxGeo g, double side, const HGeo &h, double c[3]) {
  c[0] = h.lo[0] + ((double)g.ix + 0.5) * side;
  c[1] = h.lo[1] + ((double)g.iy + 0.5) * side;
  c[2] = h.lo[2] + ((double)g.iz + 0.5) * side;
}

__global__ void k_h_gather_q(int64_t n, const int32_t *__restrict__ perm, const double2 *__restrict__ q,
                             double2 *__restrict__ qs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) qs[i] = q[perm[i]];
}

// Point-to-expansion (P2M at a leaf, P2L at a box from its X list): the
// sources are staged kHelmBatch at a time; each staged point's conj(R_n^m)
// (P2M) or h_n conj(Y_n^m) (P2L) goes to shared memory, then one thread per
// coefficient adds the batch with the weights 4 pi i kappa q_j.
template <bool LOCAL>
__global__ void __launch_bounds__(kHelmThreads)
    k_h_p2x(int p, int64_t nitems, const int32_t *__restrict__ items, const int32_t *__restrict__ xoff,
            const int32_t *__restrict__ xidx, const BoxGeo *__restrict__ geo,
            const double *__restrict__ side, const int32_t *__restrict__ first,
            const int32_t *__restrict__ count, const double *__restrict__ xyz,
            const double2 *__restrict__ q, HGeo h, double2 *__restrict__ out) {
  extern __shared__ double2 h_smem[];
  const int NC = (p + 1) * (p + 1);
  double2 *vals = h_smem;                     // [kHelmBatch][NC]
  double2 *wts = h_smem + kHelmBatch * NC;    // [kHelmBatch]
  const int64_t it = blockIdx.x;
  if (it >= nitems) return;
  const int32_t b = items[it];
  double c[3];
  box_center(geo[b], side[b], h, c);
  double2 acc[(kHelmMaxNC + kHelmThreads - 1) / kHelmThreads];
#pragma unroll
  for (int s = 0; s < (kHelmMaxNC + kHelmThreads - 1) / kHelmThreads; ++s) acc[s] = make_double2(0, 0);
  // sources: the leaf's own points (P2M) or the points of every X-list leaf (P2L)
  const int32_t e0 = LOCAL ? xoff[b] : 0, e1 = LOCAL ? xoff[b + 1] : 1;
  for (int32_t e = e0; e < e1; ++e) {
    const int32_t A = LOCAL ? xidx[e] : b;
    const int32_t f = first[A], cnt = count[A];
    for (int32_t j0 = 0; j0 < cnt; j0 += kHelmBatch) {
      const int nb = min(kHelmBatch, cnt - j0);
      if (threadIdx.x < nb) {
        const int32_t j = f + j0 + threadIdx.x;
        const double dx = xyz[3 * j] - c[0], dy = xyz[3 * j + 1] - c[1], dz = xyz[3 * j + 2] - c[2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        double jn[kHelmMaxOrder + 1], yn[kHelmMaxOrder + 1];
        if (LOCAL)
          sph_bessel<true>(p, h.kappa * r, jn, yn);
        else
          sph_bessel<false>(p, h.kappa * r, jn, yn);
        double2 *v = vals + threadIdx.x * NC;
        for_harmonics(p, dx, dy, dz, [&](int n, int m, double2 y) {
          // radial factor: j_n (P2M) or h_n (P2L), times conj(Y)
          const double2 rad = make_double2(jn[n], LOCAL ? yn[n] : 0.0);
          const double2 cy = cconj(y);
          v[hc(n, m)] = cmul(rad, cy);
          if (m > 0) {
            // conj(Y_n^{-m}) = (-1)^m Y_n^m
            const double2 ym = (m & 1) ? make_double2(-y.x, -y.y) : y;
            v[hc(n, -m)] = cmul(rad, ym);
          }
        });
        // P2M stores conj(R) = j_n conj(Y): for real j_n, conj(j_n Y) = j_n conj(Y)
        const double2 qj = q[j];
        wts[threadIdx.x] = make_double2(-4.0 * kPi * h.kappa * qj.y, 4.0 * kPi * h.kappa * qj.x);
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < (kHelmMaxNC + kHelmThreads - 1) / kHelmThreads; ++s) {
        const int cidx = threadIdx.x + s * kHelmThreads;
        if (cidx < NC)
          for (int t = 0; t < nb; ++t) acc[s] = cmad(wts[t], vals[t * NC + cidx], acc[s]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int s = 0; s < (kHelmMaxNC + kHelmThreads - 1) / kHelmThreads; ++s) {
    const int cidx = threadIdx.x + s * kHelmThreads;
    if (cidx < NC) {
      double2 *o = out + (int64_t)b * NC + cidx;
      *o = LOCAL ? cadd(*o, acc[s]) : acc[s];
    }
  }
}

// out[b] (=|+=) sum over sources s of T(s) in[s]: one CTA per box, one thread
// per output coefficient, each source's coefficients staged in shared memory.
//  MODE 0 (M2M): b a parent, sources its children, T = m2m[child octant];
//  MODE 1 (M2L): b at a level >= 2, sources its V list, T = m2l[offset code];
//  MODE 2 (L2L): b a child, source its parent, T = l2l[b's octant], added.
template <int MODE>
__global__ void __launch_bounds__(kHelmMaxNC + 23)
    k_h_translate(int p, int32_t b0, int32_t nbox, const int32_t *__restrict__ voff,
                  const int32_t *__restrict__ vidx, const int32_t *__restrict__ child,
                  const int32_t *__restrict__ nchild, const int32_t *__restrict__ parent,
                  const BoxGeo *__restrict__ geo, const double2 *__restrict__ ops,
                  const double2 *__restrict__ in, double2 *__restrict__ out) {
  __shared__ double2 s_in[kHelmMaxNC];
  const int NC = (p + 1) * (p + 1);
  const int32_t b = b0 + blockIdx.x;
  if (blockIdx.x >= nbox) return;
  const int j = threadIdx.x;
  double2 acc = make_double2(0.0, 0.0);
  int32_t ns, s0 = 0;
  if (MODE == 0) {
    ns = nchild[b];
    s0 = child[b];
    if (ns == 0) return;  // a leaf keeps the multipole of its P2M
  } else if (MODE == 1) {
    s0 = voff[b];
    ns = voff[b + 1] - s0;
  } else {
    ns = 1;
  }
  const BoxGeo gb = geo[b];
  for (int32_t t = 0; t < ns; ++t) {
    int32_t A;
    const double2 *T;
    if (MODE == 0) {
      A = s0 + t;
      const BoxGeo ga = geo[A];
      T = ops + (int64_t)((ga.ix & 1) | ((ga.iy & 1) << 1) | ((ga.iz & 1) << 2)) * NC * NC;
    } else if (MODE == 1) {
      A = vidx[s0 + t];
      const BoxGeo ga = geo[A];
      const int code = (gb.ix - ga.ix + 3) * 49 + (gb.iy - ga.iy + 3) * 7 + (gb.iz - ga.iz + 3);
      T = ops + (int64_t)code * NC * NC;
    } else {
      A = parent[b];
      T = ops + (int64_t)((gb.ix & 1) | ((gb.iy & 1) << 1) | ((gb.iz & 1) << 2)) * NC * NC;
    }
    __syncthreads();
    if (j < NC) s_in[j] = in[(int64_t)A * NC + j];
    __syncthreads();
    if (j < NC) {
      const double2 *tj = T + j;
#pragma unroll 4
      for (int k = 0; k < NC; ++k) acc = cmad(tj[(int64_t)k * NC], s_in[k], acc);
    }
  }
  if (j < NC) {
    double2 *o = out + (int64_t)b * NC + j;
    *o = MODE == 2 ? cadd(*o, acc) : acc;
  }
}

// Far field at the targets of a leaf: L2P from the leaf's local expansion and
// M2P from the multipole of every box of its W list.  One CTA per leaf, a
// thread per target; the coefficient vector in use is staged in shared memory.
__global__ void __launch_bounds__(kHelmThreads)
    k_h_far(int p, int64_t nleaves, const int32_t *__restrict__ leaves, const int32_t *__restrict__ woff,
            const int32_t *__restrict__ widx, const BoxGeo *__restrict__ geo,
            const double *__restrict__ side, const int32_t *__restrict__ first,
            const int32_t *__restrict__ count, const double *__restrict__ xyz,
            const double2 *__restrict__ M, const double2 *__restrict__ L, HGeo h,
            double2 *__restrict__ far) {
  __shared__ double2 s_c[kHelmMaxNC];
  const int NC = (p + 1) * (p + 1);
  if (blockIdx.x >= nleaves) return;
  const int32_t b = leaves[blockIdx.x];
  const int32_t f = first[b], cnt = count[b];
  const int32_t e0 = woff[b], e1 = woff[b + 1];
  const bool has_local = geo[b].level >= 2;
  for (int32_t i0 = 0; i0 < cnt; i0 += kHelmThreads) {
    const int32_t i = i0 + threadIdx.x;
    double2 acc = make_double2(0.0, 0.0);
    double tx = 0, ty = 0, tz = 0;
    if (i < cnt) {
      tx = xyz[3 * (f + i)];
      ty = xyz[3 * (f + i) + 1];
      tz = xyz[3 * (f + i) + 2];
    }
    for (int32_t e = has_local ? e0 - 1 : e0; e < e1; ++e) {
      const bool local = e < e0;  // the leaf's own local expansion first
      const int32_t A = local ? b : widx[e];
      __syncthreads();
      for (int c = threadIdx.x; c < NC; c += kHelmThreads)
        s_c[c] = local ? L[(int64_t)b * NC + c] : M[(int64_t)A * NC + c];
      __syncthreads();
      if (i >= cnt) continue;
      double c[3];
      box_center(geo[A], side[A], h, c);
      const double dx = tx - c[0], dy = ty - c[1], dz = tz - c[2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      double jn[kHelmMaxOrder + 1], yn[kHelmMaxOrder + 1];
      if (local)
        sph_bessel<false>(p, h.kappa * r, jn, yn);
      else
        sph_bessel<true>(p, h.kappa * r, jn, yn);
      for_harmonics(p, dx, dy, dz, [&](int n, int m, double2 y) {
        // sum over +-m of C_n^{+-m} Y_n^{+-m}, then times the radial factor
        double2 t = cmul(s_c[hc(n, m)], y);
        if (m > 0) {
          const double2 ym = (m & 1) ? make_double2(-y.x, y.y) : make_double2(y.x, -y.y);
          t = cmad(s_c[hc(n, -m)], ym, t);
        }
        const double2 rad = make_double2(jn[n], local ? 0.0 : yn[n]);
        acc = cmad(rad, t, acc);
      });
    }
    if (i < cnt) far[f + i] = acc;
  }
}

// Near field of a leaf's targets over its U list, plus the far field; stores
// phi at each target's input index.  One CTA per leaf; the sources of each U
// leaf are staged in shared memory, kHelmThreads at a time.
__global__ void __launch_bounds__(kHelmThreads)
    k_h_p2p(int64_t nleaves, const int32_t *__restrict__ leaves, const int32_t *__restrict__ uoff,
            const int32_t *__restrict__ uidx, const int32_t *__restrict__ first,
            const int32_t *__restrict__ count, const double *__restrict__ xyz,
            const double2 *__restrict__ q, const double2 *__restrict__ far,
            const int32_t *__restrict__ perm, double kappa, double2 *__restrict__ phi) {
  __shared__ double s_x[kHelmThreads], s_y[kHelmThreads], s_z[kHelmThreads];
  __shared__ double2 s_q[kHelmThreads];
  if (blockIdx.x >= nleaves) return;
  const int32_t b = leaves[blockIdx.x];
  const int32_t f = first[b], cnt = count[b];
  const int32_t e0 = uoff[b], e1 = uoff[b + 1];
  for (int32_t i0 = 0; i0 < cnt; i0 += kHelmThreads) {
    const int32_t i = i0 + threadIdx.x;
    double tx = 0, ty = 0, tz = 0;
    if (i < cnt) {
      tx = xyz[3 * (f + i)];
      ty = xyz[3 * (f + i) + 1];
      tz = xyz[3 * (f + i) + 2];
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t A = uidx[e];
      const int32_t fa = first[A], ca = count[A];
      for (int32_t j0 = 0; j0 < ca; j0 += kHelmThreads) {
        const int nj = min(kHelmThreads, ca - j0);
        __syncthreads();
        if (threadIdx.x < nj) {
          const int32_t j = fa + j0 + threadIdx.x;
          s_x[threadIdx.x] = xyz[3 * j];
          s_y[threadIdx.x] = xyz[3 * j + 1];
          s_z[threadIdx.x] = xyz[3 * j + 2];
          s_q[threadIdx.x] = q[j];
        }
        __syncthreads();
        if (i < cnt)
          for (int t = 0; t < nj; ++t) {
            const double dx = tx - s_x[t], dy = ty - s_y[t], dz = tz - s_z[t];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            const double r = sqrt(r2);
            double sn, cs;
            sincos(kappa * r, &sn, &cs);
            const double ir = 1.0 / r;
            acc = cmad(s_q[t], make_double2(cs * ir, sn * ir), acc);
          }
      }
    }
    if (i < cnt) phi[perm[f + i]] = cadd(far[f + i], acc);
  }
}

// M2L in FP32 (plans of mixed precision).  The coefficients of a level of
// side a are scaled by powers of s = min(kappa a, 1), as the Laplace ones are
// by powers of a: M^_n = M_n / s^n, L^_n' = L_n' s^{n'+1}, so that the
// operator T^_{n'n} = T_{n'n} s^{n+n'+1} and both vectors stay well inside the
// FP32 range at any depth (the unscaled h_l(kappa |t|) overflows it on deep
// trees).  Coefficients stay FP64 in memory; M is scaled and rounded when it
// is staged, L is unscaled in FP64 when it is stored.
__global__ void k_h_m2l_to_f32(int64_t nops, int p, double sc, const double2 *__restrict__ op,
                               float2 *__restrict__ op32) {
  const int NC = (p + 1) * (p + 1);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nops * NC * NC) return;
  const int kj = (int)(e % ((int64_t)NC * NC)), k = kj / NC, j = kj % NC;
  const int nk = (int)sqrtf((float)k + 0.5f), nj = (int)sqrtf((float)j + 0.5f);
  const double f = pow(sc, (double)(nk + nj + 1));
  const double2 v = op[e];
  op32[e] = make_float2((float)(v.x * f), (float)(v.y * f));
}

constexpr int kHelmM2LChunk = 4;  // V sources staged per barrier in the FP32 M2L

__global__ void __launch_bounds__(kHelmMaxNC + 23)
    k_h_m2l32(int p, int32_t b0, int32_t nbox, const int32_t *__restrict__ voff,
              const int32_t *__restrict__ vidx, const BoxGeo *__restrict__ geo,
              const float2 *__restrict__ ops, double sc, const double2 *__restrict__ M,
              double2 *__restrict__ L) {
  __shared__ float2 s_in[kHelmM2LChunk][kHelmMaxNC];
  __shared__ const float2 *s_op[kHelmM2LChunk];
  const int NC = (p + 1) * (p + 1);
  if (blockIdx.x >= nbox) return;
  const int32_t b = b0 + blockIdx.x;
  const int j = threadIdx.x;
  const int nj = j < NC ? (int)sqrtf((float)j + 0.5f) : 0;
  const double in_scale = pow(sc, -(double)nj);
  const int32_t s0 = voff[b], ns = voff[b + 1] - s0;
  const BoxGeo gb = geo[b];
  float2 acc = make_float2(0.f, 0.f);
  for (int32_t t0 = 0; t0 < ns; t0 += kHelmM2LChunk) {
    const int nt = min(kHelmM2LChunk, ns - t0);
    __syncthreads();
    for (int t = 0; t < nt; ++t) {
      const int32_t A = vidx[s0 + t0 + t];
      if (j < NC) {
        const double2 v = M[(int64_t)A * NC + j];
        s_in[t][j] = make_float2((float)(v.x * in_scale), (float)(v.y * in_scale));
      }
      if (j == 0) {
        const BoxGeo ga = geo[A];
        const int code = (gb.ix - ga.ix + 3) * 49 + (gb.iy - ga.iy + 3) * 7 + (gb.iz - ga.iz + 3);
        s_op[t] = ops + (int64_t)code * NC * NC;
      }
    }
    __syncthreads();
    if (j < NC)
      for (int t = 0; t < nt; ++t) {
        const float2 *tj = s_op[t] + j;
        const float2 *m = s_in[t];
#pragma unroll 4
        for (int k = 0; k < NC; ++k) {
          const float2 o = tj[(int64_t)k * NC], v = m[k];
          acc.x = fmaf(o.x, v.x, fmaf(-o.y, v.y, acc.x));
          acc.y = fmaf(o.x, v.y, fmaf(o.y, v.x, acc.y));
        }
      }
  }
  if (j < NC) {
    const double out_scale = pow(sc, -(double)(nj + 1));
    L[(int64_t)b * NC + j] = make_double2((double)acc.x * out_scale, (double)acc.y * out_scale);
  }
}

// The near field in FP32 (plans of mixed precision): the sources of each U
// leaf are staged in the target leaf's frame (x_j - c_B, from the FP64 leaf
// offsets, rounded once), e^{i kappa r}/r is evaluated with sincosf and rsqrt,
// and each staged batch's FP32 sum is added to an FP64 total.
__device__ __forceinline__ double center_off(int32_t ia, double sa, int32_t ib, double sb) {
  return ((double)ia + 0.5) * sa - ((double)ib + 0.5) * sb;
}

__global__ void __launch_bounds__(kHelmThreads)
    k_h_p2p32(int64_t nleaves, const int32_t *__restrict__ leaves, const int32_t *__restrict__ uoff,
              const int32_t *__restrict__ uidx, const int32_t *__restrict__ first,
              const int32_t *__restrict__ count, const BoxGeo *__restrict__ geo,
              const double *__restrict__ side, const Dbl4 *__restrict__ pl,
              const double2 *__restrict__ q, const double2 *__restrict__ far,
              const int32_t *__restrict__ perm, float kappa, double2 *__restrict__ phi) {
  __shared__ float4 s_p[kHelmThreads];  // x, y, z, Re q
  __shared__ float s_qi[kHelmThreads];  // Im q
  if (blockIdx.x >= nleaves) return;
  const int32_t b = leaves[blockIdx.x];
  const int32_t f = first[b], cnt = count[b];
  const int32_t e0 = uoff[b], e1 = uoff[b + 1];
  const BoxGeo gb = geo[b];
  const double sb = side[b];
  for (int32_t i0 = 0; i0 < cnt; i0 += kHelmThreads) {
    const int32_t i = i0 + threadIdx.x;
    float tx = 0.f, ty = 0.f, tz = 0.f;
    if (i < cnt) {
      const Dbl4 t = pl[f + i];
      tx = (float)t.x;
      ty = (float)t.y;
      tz = (float)t.z;
    }
    double accr = 0.0, acci = 0.0;
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t A = uidx[e];
      const int32_t fa = first[A], ca = count[A];
      const BoxGeo ga = geo[A];
      const double sa = side[A];
      const double ox = center_off(ga.ix, sa, gb.ix, sb), oy = center_off(ga.iy, sa, gb.iy, sb),
                   oz = center_off(ga.iz, sa, gb.iz, sb);
      for (int32_t j0 = 0; j0 < ca; j0 += kHelmThreads) {
        const int nj = min(kHelmThreads, ca - j0);
        __syncthreads();
        if (threadIdx.x < nj) {
          const int32_t j = fa + j0 + threadIdx.x;
          const Dbl4 v = pl[j];
          const double2 qj = q[j];
          s_p[threadIdx.x] = make_float4((float)(v.x + ox), (float)(v.y + oy), (float)(v.z + oz),
                                         (float)qj.x);
          s_qi[threadIdx.x] = (float)qj.y;
        }
        __syncthreads();
        if (i < cnt) {
          float sr = 0.f, si = 0.f;
          for (int t = 0; t < nj; ++t) {
            const float4 sp = s_p[t];
            const float dx = tx - sp.x, dy = ty - sp.y, dz = tz - sp.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 == 0.f) continue;
            const float ir = rsqrtf(r2);
            float sn, cs;
            sincosf(kappa * (r2 * ir), &sn, &cs);
            const float gr = cs * ir, gi = sn * ir, qi = s_qi[t];
            sr = fmaf(sp.w, gr, fmaf(-qi, gi, sr));
            si = fmaf(sp.w, gi, fmaf(qi, gr, si));
          }
          accr += (double)sr;
          acci += (double)si;
        }
      }
    }
    if (i < cnt) {
      const double2 fr = far[f + i];
      phi[perm[f + i]] = make_double2(fr.x + accr, fr.y + acci);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

using cd = std::complex<double>;

// Once per device (constant memory and kernel attributes belong to a
// device): the recurrence constants of the harmonics, and the dynamic
// shared-memory limit of the P2M / P2L kernels.  Synchronous the first time.
void device_setup() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  for (int d : done)
    if (d == dev) return;
  double sec[kHelmMaxOrder + 1] = {}, fst[kHelmMaxOrder + 1] = {}, a[kHelmMaxNC] = {},
         b[kHelmMaxNC] = {};
  for (int m = 1; m <= kHelmMaxOrder; ++m) sec[m] = -std::sqrt((2.0 * m + 1.0) / (2.0 * m));
  for (int m = 0; m <= kHelmMaxOrder; ++m) fst[m] = std::sqrt(2.0 * m + 3.0);
  for (int n = 2; n <= kHelmMaxOrder; ++n)
    for (int m = 0; m <= n - 2; ++m) {
      a[hc(n, m)] = std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
      b[hc(n, m)] = std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
    }
  FMM_CUDA(cudaMemcpyToSymbol(c_sec, sec, sizeof(sec)));
  FMM_CUDA(cudaMemcpyToSymbol(c_first, fst, sizeof(fst)));
  FMM_CUDA(cudaMemcpyToSymbol(c_a, a, sizeof(a)));
  FMM_CUDA(cudaMemcpyToSymbol(c_b, b, sizeof(b)));
  const int mx = (kHelmBatch * kHelmMaxNC + kHelmBatch) * (int)sizeof(double2);
  FMM_CUDA(cudaFuncSetAttribute(k_h_p2x<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  FMM_CUDA(cudaFuncSetAttribute(k_h_p2x<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
  done.push_back(dev);
}

// Y_n^m(d^) for n <= P, all m (the device recurrence, with its constants
// computed in place)
void host_harmonics(int P, const double d[3], std::vector<cd> &Y) {
  Y.assign((size_t)(P + 1) * (P + 1), cd(0, 0));
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double u = 1.0;
  cd w(0, 0);
  if (r2 > 0.0) {
    const double ir = 1.0 / std::sqrt(r2);
    u = d[2] * ir;
    w = cd(d[0] * ir, d[1] * ir);
  }
  cd ymm(0.28209479177387814347403972578038629, 0.0);
  for (int m = 0; m <= P; ++m) {
    if (m > 0) ymm = -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * w * ymm;
    Y[(size_t)hc(m, m)] = ymm;
    if (m < P) {
      cd y2 = ymm, y1 = std::sqrt(2.0 * m + 3.0) * u * ymm;
      Y[(size_t)hc(m + 1, m)] = y1;
      for (int n = m + 2; n <= P; ++n) {
        const double a = std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
        const double b = std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
        const cd y0 = a * (u * y1 - b * y2);
        Y[(size_t)hc(n, m)] = y0;
        y2 = y1;
        y1 = y0;
      }
    }
    for (int n = m; n <= P && m > 0; ++n)
      Y[(size_t)hc(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(Y[(size_t)hc(n, m)]);
  }
}

// Gaunt table for n, n' <= p: entry (k * NC + j) * (p + 1) + (l - |n - n'|)/2,
// G = 2 pi int_{-1}^{1} Y_n^m(t,0) Y_n'^m'(t,0) Y_l^{m-m'}(t,0) d(cos t) by a
// Gauss-Legendre rule of 2p + 2 nodes (exact: the integrand is a polynomial of
// degree n + n' + l <= 4p in cos t).  Nodes by Newton's method on P_{2p+2}.
std::vector<double> host_gaunt(int p) {
  const int nq = 2 * p + 2, NC = (p + 1) * (p + 1), P2 = 2 * p;
  std::vector<double> xs(nq), ws(nq);
  for (int k = 0; k < nq; ++k) {
    double x = std::cos(kPi * (k + 0.75) / (nq + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int m = 2; m <= nq; ++m) {
        const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      dp = nq * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) {
        // one more derivative at the converged node
        p0 = 1.0;
        p1 = x;
        for (int m = 2; m <= nq; ++m) {
          const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
          p0 = p1;
          p1 = p2;
        }
        dp = nq * (x * p1 - p0) / (x * x - 1.0);
        break;
      }
    }
    xs[k] = x;
    ws[k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  const int N2 = (P2 + 1) * (P2 + 1);
  std::vector<double> T((size_t)nq * N2);
  std::vector<cd> Y;
  for (int k = 0; k < nq; ++k) {
    const double d[3] = {std::sqrt(std::max(0.0, 1.0 - xs[k] * xs[k])), 0.0, xs[k]};
    host_harmonics(P2, d, Y);
    for (int c = 0; c < N2; ++c) T[(size_t)k * N2 + c] = Y[(size_t)c].real();
  }
  std::vector<double> G((size_t)NC * NC * (p + 1), 0.0);
  for (int n = 0; n <= p; ++n)
    for (int m = -n; m <= n; ++m)
      for (int n2 = 0; n2 <= p; ++n2)
        for (int m2 = -n2; m2 <= n2; ++m2) {
          const int mu = m - m2, l0 = std::abs(n - n2);
          for (int l = l0; l <= n + n2; l += 2) {
            if (std::abs(mu) > l) continue;
            double s = 0.0;
            for (int k = 0; k < nq; ++k)
              s += ws[k] * T[(size_t)k * N2 + hc(n, m)] * T[(size_t)k * N2 + hc(n2, m2)] *
                   T[(size_t)k * N2 + hc(l, mu)];
            G[((size_t)hc(n, m) * NC + hc(n2, m2)) * (p + 1) + (l - l0) / 2] = 2.0 * kPi * s;
          }
        }
  return G;
}

// X_l^mu(t), l <= 2p, appended to xt: R (regular) or S (singular)
void host_wave(int p, double kappa, const double t[3], bool singular, std::vector<cd> &xt) {
  const int P2 = 2 * p;
  const double r = std::sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
  double jn[2 * kHelmMaxOrder + 1], yn[2 * kHelmMaxOrder + 1];
  if (singular)
    sph_bessel<true>(P2, kappa * r, jn, yn);
  else
    sph_bessel<false>(P2, kappa * r, jn, yn);
  std::vector<cd> Y;
  host_harmonics(P2, t, Y);
  for (int l = 0; l <= P2; ++l)
    for (int mu = -l; mu <= l; ++mu)
      xt.push_back(cd(jn[l], singular ? yn[l] : 0.0) * Y[(size_t)hc(l, mu)]);
}

}  // namespace

// Operators for (kappa, p) on the plan's levels (rebuilt when kappa, p, the
// root cube or the depth change).
// scale of the FP32 M2L coefficients at a level of side a
static double helm_scale(double kappa, double a) { return std::min(kappa * a, 1.0); }

static void build_helmholtz_operators(fmm_plan_impl &P, double kappa, int p) {
  HelmholtzState &H = P.helm;
  const int nl = P.nlevels;
  const bool f32 = P.precision != FMM_FP64;
  if (H.order == p && H.kappa == kappa && H.D == P.D && H.nlevels == nl && H.f32 == f32) return;
  cudaStream_t s = P.stream;
  const int NC = (p + 1) * (p + 1), NX = (2 * p + 1) * (2 * p + 1);
  const std::vector<double> G = host_gaunt(p);
  H.gaunt.resize(G.size(), s);
  FMM_CUDA(cudaMemcpyAsync(H.gaunt.p, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  const size_t per = (size_t)NC * NC;
  H.m2l.resize((size_t)std::max(nl - 2, 1) * 343 * per, s);
  H.m2m.resize((size_t)std::max(nl, 1) * 8 * per, s);
  H.l2l.resize((size_t)std::max(nl, 1) * 8 * per, s);
  if (f32) H.m2l32.resize((size_t)std::max(nl - 2, 1) * 343 * per, s);
  std::vector<cd> xt;
  auto assemble = [&](int64_t nops, double2 *dst) {
    H.xtab.resize(xt.size(), s);
    FMM_CUDA(cudaMemcpyAsync(H.xtab.p, xt.data(), xt.size() * sizeof(cd), cudaMemcpyHostToDevice, s));
    const int64_t tot = nops * (int64_t)per;
    k_h_assemble<<<ceil_div(tot, 256), 256, 0, s>>>(nops, p, H.xtab.p, H.gaunt.p, dst);
    FMM_LAUNCH_CHECK();
    // the host table is reused for the next set: wait for this copy
    FMM_CUDA(cudaStreamSynchronize(s));
  };
  for (int l = 0; l < nl; ++l) {
    const double a = box_side(P.D, l);
    if (l >= 2) {
      xt.clear();
      for (int code = 0; code < 343; ++code) {
        const int dx = code / 49 - 3, dy = code / 7 % 7 - 3, dz = code % 7 - 3;
        if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) {
          xt.insert(xt.end(), (size_t)NX, cd(0, 0));
          continue;
        }
        const double t[3] = {dx * a, dy * a, dz * a};
        host_wave(p, kappa, t, true, xt);
      }
      assemble(343, H.m2l.p + (size_t)(l - 2) * 343 * per);
      if (f32) {
        const int64_t tot = 343 * (int64_t)per;
        k_h_m2l_to_f32<<<ceil_div(tot, 256), 256, 0, s>>>(343, p, helm_scale(kappa, a),
                                                          H.m2l.p + (size_t)(l - 2) * 343 * per,
                                                          H.m2l32.p + (size_t)(l - 2) * 343 * per);
        FMM_LAUNCH_CHECK();
      }
    }
    if (l >= 1) {
      // child octant o: child centre - parent centre = (bit - 1/2) a per axis
      for (int dir = 0; dir < 2; ++dir) {
        if (dir == 1 && l < 3) continue;
        xt.clear();
        for (int o = 0; o < 8; ++o) {
          const double h[3] = {((o & 1) - 0.5) * a, (((o >> 1) & 1) - 0.5) * a, (((o >> 2) & 1) - 0.5) * a};
          // M2M: t = c_parent - c_child; L2L: t = c_child - c_parent
          const double t[3] = {dir == 0 ? -h[0] : h[0], dir == 0 ? -h[1] : h[1], dir == 0 ? -h[2] : h[2]};
          host_wave(p, kappa, t, false, xt);
        }
        assemble(8, (dir == 0 ? H.m2m.p : H.l2l.p) + (size_t)l * 8 * per);
      }
    }
  }
  H.order = p;
  H.kappa = kappa;
  H.D = P.D;
  H.nlevels = nl;
  H.f32 = f32;
}

void eval_helmholtz(fmm_plan_impl &P, double kappa, int p, const double *d_q, double *d_phi) {
  if (P.dual) throw Error(FMM_ERR_INVALID_ARG, "the Helmholtz mat-vec needs a U/V/W/X-list plan");
  if (P.nproblems != 1) throw Error(FMM_ERR_INVALID_ARG, "the Helmholtz mat-vec takes one problem");
  if (p < 0 || p > kHelmMaxOrder) throw Error(FMM_ERR_INVALID_ARG, "Helmholtz order out of range");
  if (!(kappa > 0.0) || !std::isfinite(kappa))
    throw Error(FMM_ERR_INVALID_ARG, "kappa must be positive and finite");
  const int64_t n = P.n;
  if (n == 0) return;
  cudaStream_t s = P.stream;
  device_setup();
  if (!P.v_built) build_vlists(P);
  build_helmholtz_operators(P, kappa, p);
  HelmholtzState &H = P.helm;
  const int NC = (p + 1) * (p + 1);
  const int64_t nb = P.nboxes;
  H.M.resize((size_t)nb * NC, s);
  H.L.resize((size_t)nb * NC, s);
  H.q.resize((size_t)n, s);
  H.far.resize((size_t)n, s);
  FMM_CUDA(cudaMemsetAsync(H.L.p, 0, H.L.bytes(), s));
  HGeo hg;
  hg.lo[0] = P.lo[0];
  hg.lo[1] = P.lo[1];
  hg.lo[2] = P.lo[2];
  hg.kappa = kappa;
  const double2 *q = reinterpret_cast<const double2 *>(d_q);
  double2 *phi = reinterpret_cast<double2 *>(d_phi);
  k_h_gather_q<<<ceil_div(n, 256), 256, 0, s>>>(n, P.perm.p, q, H.q.p);
  FMM_LAUNCH_CHECK();
  const size_t smem = (size_t)(kHelmBatch * NC + kHelmBatch) * sizeof(double2);
  {
    PassScope ps(P, kPassP2M);
    k_h_p2x<false><<<(unsigned)P.nleaves, kHelmThreads, smem, s>>>(
        p, P.nleaves, P.leaves.p, nullptr, nullptr, P.box_geo.p, P.box_side.p, P.box_first.p,
        P.box_count.p, P.xyz_sorted.p, H.q.p, hg, H.M.p);
    FMM_LAUNCH_CHECK();
  }
  const int tpb = (NC + 31) / 32 * 32;
  const size_t per = (size_t)NC * NC;
  {
    PassScope ps(P, kPassM2M);
    for (int l = P.nlevels - 2; l >= 0; --l) {
      const int32_t b0 = P.level_off[l], cnt = P.level_off[l + 1] - b0;
      if (cnt == 0) continue;
      k_h_translate<0><<<cnt, tpb, 0, s>>>(p, b0, cnt, nullptr, nullptr, P.box_child.p,
                                           P.box_nchild.p, nullptr, P.box_geo.p,
                                           H.m2m.p + (size_t)(l + 1) * 8 * per, H.M.p, H.M.p);
      FMM_LAUNCH_CHECK();
    }
  }
  {
    PassScope ps(P, kPassM2L);
    for (int l = 2; l < P.nlevels; ++l) {
      const int32_t b0 = P.level_off[l], cnt = P.level_off[l + 1] - b0;
      if (cnt == 0) continue;
      if (H.f32)
        k_h_m2l32<<<cnt, tpb, 0, s>>>(p, b0, cnt, P.v_off.p, P.v_idx.p, P.box_geo.p,
                                      H.m2l32.p + (size_t)(l - 2) * 343 * per,
                                      helm_scale(kappa, box_side(P.D, l)), H.M.p, H.L.p);
      else
        k_h_translate<1><<<cnt, tpb, 0, s>>>(p, b0, cnt, P.v_off.p, P.v_idx.p, nullptr, nullptr,
                                             nullptr, P.box_geo.p, H.m2l.p + (size_t)(l - 2) * 343 * per,
                                             H.M.p, H.L.p);
      FMM_LAUNCH_CHECK();
    }
  }
  if (P.nxboxes > 0) {
    PassScope ps(P, kPassP2L);
    k_h_p2x<true><<<(unsigned)P.nxboxes, kHelmThreads, smem, s>>>(
        p, P.nxboxes, P.xboxes.p, P.x_off.p, P.x_idx.p, P.box_geo.p, P.box_side.p, P.box_first.p,
        P.box_count.p, P.xyz_sorted.p, H.q.p, hg, H.L.p);
    FMM_LAUNCH_CHECK();
  }
  {
    PassScope ps(P, kPassL2L);
    for (int l = 3; l < P.nlevels; ++l) {
      const int32_t b0 = P.level_off[l], cnt = P.level_off[l + 1] - b0;
      if (cnt == 0) continue;
      k_h_translate<2><<<cnt, tpb, 0, s>>>(p, b0, cnt, nullptr, nullptr, nullptr, nullptr,
                                           P.box_parent.p, P.box_geo.p, H.l2l.p + (size_t)l * 8 * per,
                                           H.L.p, H.L.p);
      FMM_LAUNCH_CHECK();
    }
  }
  {
    PassScope ps(P, kPassL2P);
    k_h_far<<<(unsigned)P.nleaves, kHelmThreads, 0, s>>>(
        p, P.nleaves, P.leaves.p, P.w_off.p, P.w_idx.p, P.box_geo.p, P.box_side.p, P.box_first.p,
        P.box_count.p, P.xyz_sorted.p, H.M.p, H.L.p, hg, H.far.p);
    FMM_LAUNCH_CHECK();
  }
  {
    PassScope ps(P, kPassP2P);
    if (P.precision == FMM_FP64)
      k_h_p2p<<<(unsigned)P.nleaves, kHelmThreads, 0, s>>>(
          P.nleaves, P.leaves.p, P.u_off.p, P.u_idx.p, P.box_first.p, P.box_count.p, P.xyz_sorted.p,
          H.q.p, H.far.p, P.perm.p, kappa, phi);
    else
      k_h_p2p32<<<(unsigned)P.nleaves, kHelmThreads, 0, s>>>(
          P.nleaves, P.leaves.p, P.u_off.p, P.u_idx.p, P.box_first.p, P.box_count.p, P.box_geo.p,
          P.box_side.p, P.pl64.p, H.q.p, H.far.p, P.perm.p, (float)kappa, phi);
    FMM_LAUNCH_CHECK();
  }
}

void release_helmholtz(fmm_plan_impl &P) {
  HelmholtzState &H = P.helm;
  H.gaunt.release();
  H.m2l.release();
  H.m2m.release();
  H.l2l.release();
  H.m2l32.release();
  H.xtab.release();
  H.M.release();
  H.L.release();
  H.q.release();
  H.far.release();
  H.order = -1;
}

}  // namespace fmm

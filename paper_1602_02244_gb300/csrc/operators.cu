// operators.cu -- precomputed translation matrices (§2.2: translation
// operators are matrices acting on coefficient vectors; translational
// invariance gives O(1) distinct operators per level, and with scale-free
// coefficients one set serves every level).
//
// Basis: complex solid harmonics with Condon-Shortley phase,
//   R_n^m = r^n P_n^m(cos t) e^{imp} / (n+m)!,  I_n^m = (n-m)! P_n^m e^{imp} / r^{n+1},
// X_n^{-m} = (-1)^m conj(X_n^m).  For real charges the coefficients obey the
// same symmetry, so a box stores (p+1)^2 reals: slot n^2+n+m holds Re X_n^m
// (m >= 0) and slot n^2+n-m holds Im X_n^m (m > 0).
// Scale-free coefficients at a level of side a: M^_n = M_n / a^n,
// L^_n = L_n a^{n+1}.  Then (addition theorem of the solid harmonics)
//   M2L(d): L^_n^m = (-1)^{n+m} sum_{k,l} M^_k^l I_{n+k}^{l-m}(d)   d = (c_B - c_A)/a
//   M2M(h): M^_n^m(P) = 2^{-n} sum_{k,l} conj(R_{n-k}^{m-l}(h)) M^_k^l(C)
//   L2L(h): L^_k^l(C) = sum_{n,m} 2^{-(n+1)} R_{n-k}^{m-l}(h) L^_n^m(P)
// with h = (c_C - c_P)/a_C = (+-1/2, +-1/2, +-1/2) for the child's octant.
// Built once per order on the host in FP64 and kept on the device in FP64
// and FP32.
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "m2l_config.cuh"
#include "plan.cuh"

namespace fmm {

namespace {

using cd = std::complex<double>;

// Harmonic table over the full range -n <= m <= n, n <= p.
struct Harm {
  int p;
  std::vector<cd> v;
  explicit Harm(int p_) : p(p_), v((size_t)ncoef(p_)) {}
  cd get(int n, int m) const {
    if (n < 0 || n > p || m > n || -m > n) return cd(0, 0);
    return v[(size_t)cidx(n, m)];
  }
};

void fill_negative(Harm &h) {
  for (int n = 1; n <= h.p; ++n)
    for (int m = 1; m <= n; ++m)
      h.v[(size_t)cidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * std::conj(h.v[(size_t)cidx(n, m)]);
}

Harm regular(int p, double x, double y, double z) {
  Harm h(p);
  const double rr = x * x + y * y + z * z;
  const cd w(x, y);
  cd diag(1, 0);
  for (int m = 0; m <= p; ++m) {
    if (m > 0) diag *= -w / (2.0 * m);
    cd prev(0, 0), cur = diag;
    h.v[(size_t)cidx(m, m)] = cur;
    for (int n = m + 1; n <= p; ++n) {
      cd next = ((2.0 * n - 1.0) * z * cur - rr * prev) / (double)((n - m) * (n + m));
      prev = cur;
      cur = next;
      h.v[(size_t)cidx(n, m)] = cur;
    }
  }
  fill_negative(h);
  return h;
}

Harm irregular(int p, double x, double y, double z) {
  Harm h(p);
  const double rr = x * x + y * y + z * z;
  const double inv = 1.0 / rr;
  const cd w(x, y);
  cd diag(1.0 / std::sqrt(rr), 0);
  for (int m = 0; m <= p; ++m) {
    if (m > 0) diag *= -(2.0 * m - 1.0) * w * inv;
    cd prev(0, 0), cur = diag;
    h.v[(size_t)cidx(m, m)] = cur;
    for (int n = m + 1; n <= p; ++n) {
      cd next = ((2.0 * n - 1.0) * z * cur - ((double)(n - 1) * (n - 1) - (double)m * m) * prev) * inv;
      prev = cur;
      cur = next;
      h.v[(size_t)cidx(n, m)] = cur;
    }
  }
  fill_negative(h);
  return h;
}

// Real matrix (row-major [out][in]) of an R-linear map given by its complex
// matrix C[(n,m)][(k,l)] over the full index range.
template <typename F>
void realify(int p, F &&C, double *out) {
  const int nc = ncoef(p);
  for (int k = 0; k <= p; ++k)
    for (int l = 0; l <= k; ++l) {
      const double s = (l & 1) ? -1.0 : 1.0;
      for (int part = 0; part < (l == 0 ? 1 : 2); ++part) {
        // part 0: unit real part (X_k^l = 1, X_k^{-l} = s); part 1: unit
        // imaginary part (X_k^l = i, X_k^{-l} = -s i)
        const int col = part == 0 ? cidx(k, l) : cidx(k, -l);
        for (int n = 0; n <= p; ++n)
          for (int m = 0; m <= n; ++m) {
            cd y;
            if (l == 0) y = C(n, m, k, 0);
            else if (part == 0) y = C(n, m, k, l) + s * C(n, m, k, -l);
            else y = cd(0, 1) * (C(n, m, k, l) - s * C(n, m, k, -l));
            out[(size_t)cidx(n, m) * nc + col] = y.real();
            if (m > 0) out[(size_t)cidx(n, -m) * nc + col] = y.imag();
          }
      }
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the three-term
// recurrence of the Legendre polynomials)
void gauss_legendre(int N, std::vector<double> &x, std::vector<double> &w) {
  x.assign(N, 0.0);
  w.assign(N, 0.0);
  for (int i = 0; i < N; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (N + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= N; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (N == 1) p0 = 1.0;
      const double pn = N == 0 ? 1.0 : p1, pm = N == 1 ? 1.0 : p0;
      dp = N * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Rotated M2L (§2.2 translation operators, the O(p^3) factorisation): for
// the offset d, a rotation Q with Q d = |d| z; the multipole is re-expressed
// in the rotated frame (M' = A M, from sum M I(y) = sum M' I(Q y)), translated
// along z (only equal orders couple: L'_n^m = (-1)^{n+m} sum_k M'_k^m
// (n+k)! / |d|^{n+k+1}), and the local is re-expressed back (L = B L', from
// sum L R(y) = sum L' R(Q y)).  A and B act degree by degree; their entries
// are projections onto the harmonics of one degree, computed exactly with a
// product quadrature on the unit sphere (Gauss-Legendre in cos t, uniform
// in the azimuth), using that the degree-n harmonics are orthogonal there
// with |I_n^m|^2 integrating to 4 pi (n-m)!(n+m)!/(2n+1) and |R_n^m|^2 to
// 4 pi / ((2n+1)(n-m)!(n+m)!).
struct RotTables {
  std::vector<double> rot, zt;
};

RotTables rotation_tables(int p) {
  const int nc = ncoef(p);
  const size_t nrot = rotation_entries(p);
  RotTables t;
  t.rot.assign((size_t)343 * 2 * nrot, 0.0);
  t.zt.assign((size_t)343 * (p + 1) * (p + 1), 0.0);
  std::vector<double> fact(2 * p + 2, 1.0);
  for (int i = 1; i < (int)fact.size(); ++i) fact[i] = fact[i - 1] * i;
  std::vector<double> full((size_t)nc * nc);
  std::vector<std::vector<cd>> A(p + 1), B(p + 1);
  for (int dx = -3; dx <= 3; ++dx)
    for (int dy = -3; dy <= 3; ++dy)
      for (int dz = -3; dz <= 3; ++dz) {
        if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
        const int code = (dx + 3) * 49 + (dy + 3) * 7 + (dz + 3);
        const double dn = std::sqrt((double)(dx * dx + dy * dy + dz * dz));
        // rows of Q: e1, e2, u with u = d / |d|
        const double u[3] = {dx / dn, dy / dn, dz / dn};
        double a[3] = {1.0, 0.0, 0.0};
        if (std::fabs(u[0]) >= 0.9) a[0] = 0.0, a[1] = 1.0;
        const double au = a[0] * u[0] + a[1] * u[1] + a[2] * u[2];
        double e1[3] = {a[0] - au * u[0], a[1] - au * u[1], a[2] - au * u[2]};
        const double e1n = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (double &v : e1) v /= e1n;
        const double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2],
                              u[0] * e1[1] - u[1] * e1[0]};
        const double Q[3][3] = {{e1[0], e1[1], e1[2]}, {e2[0], e2[1], e2[2]}, {u[0], u[1], u[2]}};
        for (int n = 0; n <= p; ++n) {
          const int w = 2 * n + 1;
          A[n].assign((size_t)w * w, cd(0, 0));
          B[n].assign((size_t)w * w, cd(0, 0));
          std::vector<double> gx, gw;
          gauss_legendre(n + 1, gx, gw);
          for (int i = 0; i <= n; ++i)
            for (int j = 0; j < w; ++j) {
              const double st = std::sqrt(std::max(0.0, 1.0 - gx[i] * gx[i]));
              const double ph = 2.0 * M_PI * j / w;
              const double v[3] = {st * std::cos(ph), st * std::sin(ph), gx[i]};
              const double wt = gw[i] * 2.0 * M_PI / w;
              double qv[3], qtv[3];  // Q v and Q^T v
              for (int r = 0; r < 3; ++r) {
                qv[r] = Q[r][0] * v[0] + Q[r][1] * v[1] + Q[r][2] * v[2];
                qtv[r] = Q[0][r] * v[0] + Q[1][r] * v[1] + Q[2][r] * v[2];
              }
              const Harm Iv = irregular(n, v[0], v[1], v[2]), Iq = irregular(n, qtv[0], qtv[1], qtv[2]);
              const Harm Rv = regular(n, v[0], v[1], v[2]), Rq = regular(n, qv[0], qv[1], qv[2]);
              for (int m = -n; m <= n; ++m)
                for (int k = -n; k <= n; ++k) {
                  A[n][(size_t)(m + n) * w + (k + n)] += wt * std::conj(Iv.get(n, m)) * Iq.get(n, k);
                  B[n][(size_t)(m + n) * w + (k + n)] += wt * std::conj(Rv.get(n, m)) * Rq.get(n, k);
                }
            }
          for (int m = -n; m <= n; ++m) {
            const double ca = (2.0 * n + 1.0) / (4.0 * M_PI * fact[n - m] * fact[n + m]);
            const double cb = (2.0 * n + 1.0) * fact[n - m] * fact[n + m] / (4.0 * M_PI);
            for (int k = -n; k <= n; ++k) {
              A[n][(size_t)(m + n) * w + (k + n)] *= ca;
              B[n][(size_t)(m + n) * w + (k + n)] *= cb;
            }
          }
        }
        for (int half = 0; half < 2; ++half) {
          std::fill(full.begin(), full.end(), 0.0);
          realify(p, [&](int n, int m, int k, int l) -> cd {
            if (n != k) return cd(0, 0);
            return (half == 0 ? A : B)[n][(size_t)(m + n) * (2 * n + 1) + (l + n)];
          }, full.data());
          double *dst = t.rot.data() + ((size_t)code * 2 + half) * nrot;
          for (int n = 0; n <= p; ++n) {
            const int w = 2 * n + 1, b = n * n;
            const size_t off = (size_t)n * (2 * n - 1) * (2 * n + 1) / 3;
            for (int r = 0; r < w; ++r)
              for (int c = 0; c < w; ++c) dst[off + (size_t)r * w + c] = full[(size_t)(b + r) * nc + (b + c)];
          }
        }
        double *z = t.zt.data() + (size_t)code * (p + 1) * (p + 1);
        for (int n = 0; n <= p; ++n)
          for (int k = 0; k <= p; ++k) z[n * (p + 1) + k] = fact[n + k] / std::pow(dn, n + k + 1);
      }
  return t;
}

}  // namespace

size_t rotation_entries(int p) { return (size_t)(p + 1) * (2 * p + 1) * (2 * p + 3) / 3; }

void build_rotation(fmm_plan_impl &P) {
  const int p = P.order;
  if (!P.m2l_rot || P.ops.rot_order == p) return;
  static std::mutex mu;
  static std::map<int, RotTables> cache;  // host tables per order, built once per process
  const RotTables *t = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(p);
    if (it == cache.end()) it = cache.emplace(p, rotation_tables(p)).first;
    t = &it->second;
  }
  cudaStream_t s = P.stream;
  P.ops.rot64.resize(t->rot.size(), s);
  P.ops.zt64.resize(t->zt.size(), s);
  P.ops.rot32.resize(t->rot.size(), s);
  P.ops.zt32.resize(t->zt.size(), s);
  FMM_CUDA(cudaMemcpyAsync(P.ops.rot64.p, t->rot.data(), t->rot.size() * sizeof(double),
                           cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.ops.zt64.p, t->zt.data(), t->zt.size() * sizeof(double),
                           cudaMemcpyHostToDevice, s));
  std::vector<float> r32(t->rot.begin(), t->rot.end()), z32(t->zt.begin(), t->zt.end());
  FMM_CUDA(cudaMemcpyAsync(P.ops.rot32.p, r32.data(), r32.size() * sizeof(float),
                           cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.ops.zt32.p, z32.data(), z32.size() * sizeof(float),
                           cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaStreamSynchronize(s));  // r32 / z32 are host temporaries
  P.ops.rot_order = p;
}

void build_operators(fmm_plan_impl &P) {
  const int p = P.order;
  if (P.ops.order == p) return;
  const int nc = ncoef(p);
  const size_t nn = (size_t)nc * nc;
  std::vector<double> m2l(343 * nn, 0.0), m2m(8 * nn, 0.0), l2l(8 * nn, 0.0), tmp(nn);
  // M2L, stored input-major: m2l[code][in][out]
  for (int dx = -3; dx <= 3; ++dx)
    for (int dy = -3; dy <= 3; ++dy)
      for (int dz = -3; dz <= 3; ++dz) {
        if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) < 2) continue;
        const int code = (dx + 3) * 49 + (dy + 3) * 7 + (dz + 3);
        Harm I = irregular(2 * p, dx, dy, dz);
        realify(p, [&](int n, int m, int k, int l) {
          return (((n + m) & 1) ? -1.0 : 1.0) * I.get(n + k, l - m);
        }, tmp.data());
        double *dst = m2l.data() + code * nn;
        for (int r = 0; r < nc; ++r)
          for (int c = 0; c < nc; ++c) dst[(size_t)c * nc + r] = tmp[(size_t)r * nc + c];
      }
  for (int o = 0; o < 8; ++o) {
    const double hx = (o & 1) - 0.5, hy = ((o >> 1) & 1) - 0.5, hz = ((o >> 2) & 1) - 0.5;
    Harm R = regular(p, hx, hy, hz);
    realify(p, [&](int n, int m, int k, int l) {
      return std::ldexp(1.0, -n) * std::conj(R.get(n - k, m - l));
    }, m2m.data() + o * nn);
    // L2L: output (k,l) from input (n,m); in realify's naming out=(n,m), in=(k,l)
    realify(p, [&](int k, int l, int n, int m) {
      return std::ldexp(1.0, -(n + 1)) * R.get(n - k, m - l);
    }, l2l.data() + o * nn);
  }
  cudaStream_t s = P.stream;
  P.ops.m2l64.resize(m2l.size(), s);
  P.ops.m2m64.resize(m2m.size(), s);
  P.ops.l2l64.resize(l2l.size(), s);
  P.ops.m2l32.resize(m2l.size(), s);
  P.ops.m2m32.resize(m2m.size(), s);
  P.ops.l2l32.resize(l2l.size(), s);
  std::vector<float> f(m2l.size());
  auto up = [&](const std::vector<double> &h, DBuf<double> &d64, DBuf<float> &d32) {
    FMM_CUDA(cudaMemcpyAsync(d64.p, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    for (size_t i = 0; i < h.size(); ++i) f[i] = (float)h[i];
    FMM_CUDA(cudaMemcpyAsync(d32.p, f.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaStreamSynchronize(s));  // host vectors are reused
  };
  up(m2l, P.ops.m2l64, P.ops.m2l32);
  if (p <= kM2LStagedMaxOrder) {  // padded output-major FP32 copy for the staged kernel
    const int rows = m2l_rows(p), ld = coef_pitch(p);
    const size_t slab = (size_t)rows * ld;
    std::vector<float> padded(343 * slab, 0.f);
    for (int code = 0; code < 343; ++code)
      for (int r = 0; r < nc; ++r)
        for (int k = 0; k < nc; ++k)
          padded[code * slab + (size_t)r * ld + k] = (float)m2l[code * nn + (size_t)k * nc + r];
    P.ops.m2l32p.resize(padded.size(), s);
    FMM_CUDA(cudaMemcpyAsync(P.ops.m2l32p.p, padded.data(), padded.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaStreamSynchronize(s));
  }
  if (p <= kM2LStagedMaxOrder) {  // tensor-core operators: TF32 halves, core-matrix order
    std::vector<float> packed(m2l_tc_operator_floats(p));
    pack_m2l_tc_operators(p, m2l.data(), packed.data());
    P.ops.m2l_tc.resize(packed.size(), s);
    FMM_CUDA(cudaMemcpyAsync(P.ops.m2l_tc.p, packed.data(), packed.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s));
    // and the FP16 form with its power-of-two scales
    std::vector<uint16_t> packed16(m2l_tc16_operator_halves(p));
    std::vector<float> rows(m2l_rows(p)), cols(m2l_tc_pitch(p));
    pack_m2l_tc16_operators(p, m2l.data(), packed16.data(), rows.data(), cols.data());
    P.ops.m2l_tc16.resize(packed16.size(), s);
    P.ops.m2l_tc16_rows.resize(rows.size(), s);
    P.ops.m2l_tc16_cols.resize(cols.size(), s);
    FMM_CUDA(cudaMemcpyAsync(P.ops.m2l_tc16.p, packed16.data(), packed16.size() * sizeof(uint16_t),
                             cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaMemcpyAsync(P.ops.m2l_tc16_rows.p, rows.data(), rows.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaMemcpyAsync(P.ops.m2l_tc16_cols.p, cols.data(), cols.size() * sizeof(float),
                             cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaStreamSynchronize(s));
  }
  up(m2m, P.ops.m2m64, P.ops.m2m32);
  up(l2l, P.ops.l2l64, P.ops.l2l32);
  {  // transposed FP32 copies: t[o][k][r] = op[o][r][k], r padded to coef_pitch(p)
    const int ld = coef_pitch(p);
    std::vector<float> t((size_t)8 * nc * ld);
    auto tr = [&](const std::vector<double> &h, DBuf<float> &d) {
      std::fill(t.begin(), t.end(), 0.f);
      for (int o = 0; o < 8; ++o)
        for (int r = 0; r < nc; ++r)
          for (int k = 0; k < nc; ++k)
            t[((size_t)o * nc + k) * ld + r] = (float)h[(size_t)o * nn + (size_t)r * nc + k];
      d.resize(t.size(), s);
      FMM_CUDA(cudaMemcpyAsync(d.p, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, s));
      FMM_CUDA(cudaStreamSynchronize(s));  // t is reused
    };
    tr(m2m, P.ops.m2m32t);
    tr(l2l, P.ops.l2l32t);
  }
  P.ops.order = p;
}

}  // namespace fmm

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
#include <complex>
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

}  // namespace

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

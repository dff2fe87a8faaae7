// harmonics.cuh -- solid harmonics streamed in registers on the device.
//
// R_n^m(u) = r^n P_n^m(cos t) e^{imp} / (n+m)!   and
// I_n^m(u) = (n-m)! P_n^m(cos t) e^{imp} / r^{n+1}  (Condon-Shortley phase),
// generated for 0 <= m <= n <= p column by column (m outer, n inner) from
//   R_m^m = -(x+iy)/(2m) R_{m-1}^{m-1},  (n^2-m^2) R_n^m = (2n-1) z R_{n-1}^m - r^2 R_{n-2}^m
//   I_m^m = -(2m-1)(x+iy)/r^2 I_{m-1}^{m-1},
//   r^2 I_n^m = (2n-1) z I_{n-1}^m - ((n-1)^2-m^2) I_{n-2}^m,
// so only two previous values per column live in registers.  The callback
// receives (n, m, Re, Im).
#pragma once
#include "common.cuh"

namespace fmm {

// 1 / ((n-m)(n+m)) for 0 <= m < n <= 21
struct RecipTable {
  float f[22][22];
  double d[22][22];
};

constexpr RecipTable make_recip_table() {
  RecipTable t{};
  for (int n = 0; n < 22; ++n)
    for (int m = 0; m < 22; ++m) {
      double v = m < n ? 1.0 / (double)((n - m) * (n + m)) : 0.0;
      t.d[n][m] = v;
      t.f[n][m] = (float)v;
    }
  return t;
}

// one copy per translation unit that includes this header
static __constant__ RecipTable c_recip = make_recip_table();

template <typename T>
__device__ __forceinline__ T recip_nm(int n, int m);
template <>
__device__ __forceinline__ float recip_nm<float>(int n, int m) { return c_recip.f[n][m]; }
template <>
__device__ __forceinline__ double recip_nm<double>(int n, int m) { return c_recip.d[n][m]; }

template <typename T, typename F>
__device__ __forceinline__ void regular_stream(int p, T x, T y, T z, F &&f) {
  const T r2 = x * x + y * y + z * z;
  T dre = T(1), dim = T(0);
#pragma unroll
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      const T c = T(-0.5) / T(m);
      const T nre = c * (x * dre - y * dim), nim = c * (x * dim + y * dre);
      dre = nre;
      dim = nim;
    }
    f(m, m, dre, dim);
    T pre = T(0), pim = T(0), cre = dre, cim = dim;
#pragma unroll
    for (int n = m + 1; n <= p; ++n) {
      const T a = T(2 * n - 1) * z, s = recip_nm<T>(n, m);
      const T nre = (a * cre - r2 * pre) * s, nim = (a * cim - r2 * pim) * s;
      pre = cre;
      pim = cim;
      cre = nre;
      cim = nim;
      f(n, m, cre, cim);
    }
  }
}

template <typename T, typename F>
__device__ __forceinline__ void irregular_stream(int p, T x, T y, T z, F &&f) {
  const T r2 = x * x + y * y + z * z;
  const T inv = T(1) / r2;
  T dre = T(1) / sqrt(r2), dim = T(0);
#pragma unroll
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      const T c = -T(2 * m - 1) * inv;
      const T nre = c * (x * dre - y * dim), nim = c * (x * dim + y * dre);
      dre = nre;
      dim = nim;
    }
    f(m, m, dre, dim);
    T pre = T(0), pim = T(0), cre = dre, cim = dim;
#pragma unroll
    for (int n = m + 1; n <= p; ++n) {
      const T a = T(2 * n - 1) * z, b = T((n - 1) * (n - 1) - m * m);
      const T nre = (a * cre - b * pre) * inv, nim = (a * cim - b * pim) * inv;
      pre = cre;
      pim = cim;
      cre = nre;
      cim = nim;
      f(n, m, cre, cim);
    }
  }
}

// The regular stream for two points at once (the .x and .y halves), on the
// paired FP32 instructions: the same recurrence as regular_stream.
template <typename F>
__device__ __forceinline__ void regular_stream2(int p, float2 x, float2 y, float2 z, F &&f) {
  const float2 r2 = __ffma2_rn(z, z, __ffma2_rn(y, y, __fmul2_rn(x, x)));
  const float2 nr2 = make_float2(-r2.x, -r2.y);
  const float2 ny = make_float2(-y.x, -y.y);
  float2 dre = make_float2(1.f, 1.f), dim = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      const float cm = -0.5f / (float)m;
      const float2 c = make_float2(cm, cm);
      const float2 t1 = __ffma2_rn(ny, dim, __fmul2_rn(x, dre));  // x dre - y dim
      const float2 t2 = __ffma2_rn(y, dre, __fmul2_rn(x, dim));   // x dim + y dre
      dre = __fmul2_rn(c, t1);
      dim = __fmul2_rn(c, t2);
    }
    f(m, m, dre, dim);
    float2 pre = make_float2(0.f, 0.f), pim = make_float2(0.f, 0.f), cre = dre, cim = dim;
#pragma unroll
    for (int n = m + 1; n <= p; ++n) {
      const float an = (float)(2 * n - 1), sn = recip_nm<float>(n, m);
      const float2 a = __fmul2_rn(make_float2(an, an), z), s = make_float2(sn, sn);
      const float2 nre = __fmul2_rn(__ffma2_rn(nr2, pre, __fmul2_rn(a, cre)), s);
      const float2 nim = __fmul2_rn(__ffma2_rn(nr2, pim, __fmul2_rn(a, cim)), s);
      pre = cre;
      pim = cim;
      cre = nre;
      cim = nim;
      f(n, m, cre, cim);
    }
  }
}

// The irregular stream for two points at once (the .x and .y halves), on the
// paired FP32 instructions: the same recurrence as irregular_stream, two
// evaluations per instruction.  The reciprocal and reciprocal square root of
// r^2 stay scalar (IEEE division and square root).
template <typename F>
__device__ __forceinline__ void irregular_stream2(int p, float2 x, float2 y, float2 z, F &&f) {
  const float2 r2 = __ffma2_rn(z, z, __ffma2_rn(y, y, __fmul2_rn(x, x)));
  const float2 inv = make_float2(1.f / r2.x, 1.f / r2.y);
  float2 dre = make_float2(1.f / sqrtf(r2.x), 1.f / sqrtf(r2.y)), dim = make_float2(0.f, 0.f);
  const float2 ny = make_float2(-y.x, -y.y);
#pragma unroll
  for (int m = 0; m <= p; ++m) {
    if (m > 0) {
      const float cm = -(float)(2 * m - 1);
      const float2 c = __fmul2_rn(make_float2(cm, cm), inv);
      const float2 t1 = __ffma2_rn(ny, dim, __fmul2_rn(x, dre));  // x dre - y dim
      const float2 t2 = __ffma2_rn(y, dre, __fmul2_rn(x, dim));   // x dim + y dre
      dre = __fmul2_rn(c, t1);
      dim = __fmul2_rn(c, t2);
    }
    f(m, m, dre, dim);
    float2 pre = make_float2(0.f, 0.f), pim = make_float2(0.f, 0.f), cre = dre, cim = dim;
#pragma unroll
    for (int n = m + 1; n <= p; ++n) {
      const float an = (float)(2 * n - 1), nb = -(float)((n - 1) * (n - 1) - m * m);
      const float2 a = __fmul2_rn(make_float2(an, an), z), b = make_float2(nb, nb);
      const float2 nre = __fmul2_rn(__ffma2_rn(b, pre, __fmul2_rn(a, cre)), inv);
      const float2 nim = __fmul2_rn(__ffma2_rn(b, pim, __fmul2_rn(a, cim)), inv);
      pre = cre;
      pim = cim;
      cre = nre;
      cim = nim;
      f(n, m, cre, cim);
    }
  }
}

// complex coefficient X_n^m of a real-basis vector v (any -n <= m <= n;
// zero outside), using X_n^{-m} = (-1)^m conj(X_n^m)
template <typename T>
__device__ __forceinline__ void cget(const T *v, int p, int n, int m, T &re, T &im) {
  if (n < 0 || n > p || m > n || -m > n) {
    re = T(0);
    im = T(0);
    return;
  }
  if (m == 0) {
    re = v[cidx(n, 0)];
    im = T(0);
  } else if (m > 0) {
    re = v[cidx(n, m)];
    im = v[cidx(n, -m)];
  } else {
    const T s = ((-m) & 1) ? T(-1) : T(1);
    re = s * v[cidx(n, -m)];
    im = -s * v[cidx(n, m)];
  }
}

}  // namespace fmm

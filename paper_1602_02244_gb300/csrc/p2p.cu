// p2p.cu -- near field: direct Green's-function interactions of each leaf's
// targets with the points of its U list (§2.2: the dense diagonal blocks of
// the hierarchical matrix are exactly the direct operator).
//
// One warp per target leaf, no block-wide barriers.  The warp stages its
// U-list sources in a warp-private shared buffer, already shifted into the
// target leaf's local frame (offsets between box centres are exact), and
// every lane sweeps the staged sources (broadcast shared loads) for its 1-4
// targets:
//   r2 = |x_i - x_j|^2, rinv = rsqrt(r2),
//   phi += q rinv,  grad -= q rinv^3 (x_i - x_j).
// Zero distances occur only between points of the same leaf (coincident
// points share a Morton key, hence a leaf), so only the leaf's own points go
// through the masked loop (rinv = 0 at r2 = 0).  Each lane accumulates a
// staged batch in T (FP32 in mixed mode) and adds batch totals in FP64.
#include "eval_kernels.cuh"

namespace fmm {

namespace {

// One warp per CTA: a CTA's resources are released as soon as its leaf is
// done, so uneven leaf costs leave no idle warps holding an SM slot.
constexpr int kP2PWarps = 1;
constexpr int kP2PThreads = 32 * kP2PWarps;
constexpr int kP2PMinCtas = 16;  // resident CTAs per SM: caps registers at 128
constexpr int kMaxTPL = 4;  // targets per lane

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

__device__ __forceinline__ double center_delta(int32_t ia, double sa, int32_t ib, double sb) {
  return ((double)ia + 0.5) * sa - ((double)ib + 0.5) * sb;
}

// one source against the lane's TPL targets
template <typename T, int TPL, bool kMask, typename V>
__device__ __forceinline__ void interact(const V &s, const T (&x)[kMaxTPL], const T (&y)[kMaxTPL],
                                         const T (&z)[kMaxTPL], T (&acc)[kMaxTPL][4]) {
#pragma unroll
  for (int t = 0; t < TPL; ++t) {
    const T dx = x[t] - s.x, dy = y[t] - s.y, dz = z[t] - s.z;
    const T r2 = dx * dx + dy * dy + dz * dz;
    T rinv = rsqrt_t<T>(r2);
    if (kMask) rinv = r2 > T(0) ? rinv : T(0);
    const T qr = s.w * rinv;
    const T qr3 = qr * rinv * rinv;
    acc[t][0] += qr;
    acc[t][1] -= qr3 * dx;
    acc[t][2] -= qr3 * dy;
    acc[t][3] -= qr3 * dz;
  }
}

template <typename T, int TPL, typename V>
__device__ __forceinline__ void sweep(const V *ss, int j0, int j1, bool self, const T (&x)[kMaxTPL],
                                      const T (&y)[kMaxTPL], const T (&z)[kMaxTPL],
                                      T (&acc)[kMaxTPL][4]) {
  if (self) {
    for (int j = j0; j < j1; ++j) interact<T, TPL, true>(ss[j], x, y, z, acc);
  } else {
#pragma unroll 4
    for (int j = j0; j < j1; ++j) interact<T, TPL, false>(ss[j], x, y, z, acc);
  }
}

template <typename T, int CAP>
__global__ void __launch_bounds__(kP2PThreads, kP2PMinCtas)
    k_p2p(int64_t nleaves, const int32_t *__restrict__ leaves, const int32_t *__restrict__ uoff,
          const int32_t *__restrict__ uidx, const int32_t *__restrict__ first,
          const int32_t *__restrict__ count, const BoxGeo *__restrict__ geo,
          const typename V4<T>::type *__restrict__ src, const double *__restrict__ side, int64_t n,
          double *__restrict__ near) {
  using V = typename V4<T>::type;
  __shared__ V ss_all[kP2PWarps][CAP];
  __shared__ int32_t s_incl_all[kP2PWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t li = (int64_t)blockIdx.x * kP2PWarps + warp;
  if (li >= nleaves) return;  // whole warp: there are no block-wide barriers below
  V *ss = ss_all[warp];
  int32_t *s_incl = s_incl_all[warp];
  const int32_t B = leaves[li];
  const BoxGeo gb = geo[B];
  const double sb = side[B];
  const int32_t fb = first[B], cb = count[B];
  const int32_t e0 = uoff[B], e1 = uoff[B + 1];
  for (int32_t tc = 0; tc < cb; tc += 32 * kMaxTPL) {
    const int tcount = min(32 * kMaxTPL, cb - tc);
    const int tpl = (tcount + 31) / 32;
    T x[kMaxTPL], y[kMaxTPL], z[kMaxTPL];
#pragma unroll
    for (int t = 0; t < kMaxTPL; ++t) {
      const int i = lane + 32 * t;
      V v;
      v.x = v.y = v.z = v.w = T(0);
      if (i < tcount) v = src[fb + tc + i];
      x[t] = v.x;
      y[t] = v.y;
      z[t] = v.z;
    }
    double tot[kMaxTPL][4] = {};
    int32_t e = e0, off = 0;  // next source: leaf uidx[e], point `off` within it
    while (e < e1) {
      // ---- metadata of up to 32 source leaves, one per lane
      int32_t c = 0, f = 0, A = -1;
      T sx = T(0), sy = T(0), sz = T(0);
      if (e + lane < e1) {
        A = uidx[e + lane];
        const BoxGeo ga = geo[A];
        const int32_t skip = lane == 0 ? off : 0;
        f = first[A] + skip;
        c = count[A] - skip;
        const double sa = side[A];
        sx = (T)center_delta(ga.ix, sa, gb.ix, sb);
        sy = (T)center_delta(ga.iy, sa, gb.iy, sb);
        sz = (T)center_delta(ga.iz, sa, gb.iz, sb);
      }
      int32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const unsigned fit = __ballot_sync(0xffffffffu, e + lane < e1 && incl <= CAP);
      const int m = __popc(fit);  // incl is non-decreasing: the first m leaves fit
      const int npiece = m == 0 ? 1 : m;
      s_incl[lane] = m == 0 ? CAP : incl;  // m == 0: take CAP points of one oversized leaf
      __syncwarp();
      // ---- copy the points piece by piece, shifted into the target leaf's frame
      for (int k = 0; k < npiece; ++k) {
        const int32_t pf = __shfl_sync(0xffffffffu, f, k);
        const T px = __shfl_sync(0xffffffffu, sx, k);
        const T py = __shfl_sync(0xffffffffu, sy, k);
        const T pz = __shfl_sync(0xffffffffu, sz, k);
        const int32_t p0 = k > 0 ? s_incl[k - 1] : 0, p1 = s_incl[k];
        for (int idx = p0 + lane; idx < p1; idx += 32) {
          V v = src[pf + (idx - p0)];
          v.x += px;
          v.y += py;
          v.z += pz;
          ss[idx] = v;
        }
      }
      __syncwarp();
      // ---- sweep the staged sources piece by piece
      T acc[kMaxTPL][4];
#pragma unroll
      for (int t = 0; t < kMaxTPL; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = T(0);
      for (int k = 0; k < npiece; ++k) {
        const bool self = __shfl_sync(0xffffffffu, A, k) == B;
        const int32_t p0 = k > 0 ? s_incl[k - 1] : 0, p1 = s_incl[k];
        switch (tpl) {
          case 1: sweep<T, 1>(ss, p0, p1, self, x, y, z, acc); break;
          case 2: sweep<T, 2>(ss, p0, p1, self, x, y, z, acc); break;
          case 3: sweep<T, 3>(ss, p0, p1, self, x, y, z, acc); break;
          default: sweep<T, 4>(ss, p0, p1, self, x, y, z, acc); break;
        }
      }
#pragma unroll
      for (int t = 0; t < kMaxTPL; ++t)
#pragma unroll
        for (int a = 0; a < 4; ++a) tot[t][a] += (double)acc[t][a];
      if (m == 0) {
        off += CAP;
      } else {
        e += m;
        off = 0;
      }
      __syncwarp();  // the staged batch is consumed before it is overwritten
    }
#pragma unroll
    for (int t = 0; t < kMaxTPL; ++t) {
      const int i = lane + 32 * t;
      if (i < tcount) {
        const int64_t g = fb + tc + i;
        near[g] = tot[t][0];
        near[n + g] = tot[t][1];
        near[2 * n + g] = tot[t][2];
        near[3 * n + g] = tot[t][3];
      }
    }
  }
}

}  // namespace

template <typename T>
void launch_p2p(int64_t nleaves, const int32_t *leaves, const int32_t *uoff, const int32_t *uidx,
                const int32_t *first, const int32_t *count, const BoxGeo *geo,
                const typename V4<T>::type *src, const double *side, int64_t n, double *near,
                cudaStream_t s) {
  if (nleaves == 0) return;
  constexpr int CAP = sizeof(T) == 4 ? 640 : 320;  // 10 KB of staged sources per warp
  k_p2p<T, CAP><<<ceil_div(nleaves, kP2PWarps), kP2PThreads, 0, s>>>(nleaves, leaves, uoff, uidx,
                                                                      first, count, geo, src, side,
                                                                      n, near);
  FMM_LAUNCH_CHECK();
}

template void launch_p2p<float>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                const int32_t *, const int32_t *, const BoxGeo *, const float4 *,
                                const double *, int64_t, double *, cudaStream_t);
template void launch_p2p<double>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                 const int32_t *, const int32_t *, const BoxGeo *, const double4 *,
                                 const double *, int64_t, double *, cudaStream_t);

}  // namespace fmm

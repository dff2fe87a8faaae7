// p2p.cu -- near field: direct Green's-function interactions of each leaf's
// targets with the points of its U list (§2.2: the dense diagonal blocks of
// the hierarchical matrix are exactly the direct operator).
//
// One CTA per target leaf.  The U-list sources are staged in shared memory,
// already shifted into the target leaf's local frame (offsets between box
// centres are exact), so the inner loop is a flat sweep:
//   r2 = |x_i - x_j|^2, rinv = rsqrt(r2) (0 at r2 = 0),
//   phi += q rinv,  grad -= q rinv^3 (x_i - x_j).
// When a leaf has fewer than 128 targets, k = floor(128 / targets) threads
// share a target and split its sources; their partial sums are combined in
// FP64.  Within a staged batch each thread accumulates in T (FP32 in mixed
// mode); batch totals are added in FP64.
#include "eval_kernels.cuh"

namespace fmm {

namespace {

constexpr int kP2PThreads = 128;

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

__device__ __forceinline__ double center_delta(int32_t ia, int la, int32_t ib, int lb, double D) {
  return ((double)ia + 0.5) * box_side(D, la) - ((double)ib + 0.5) * box_side(D, lb);
}

template <typename T, int CAP>
__global__ void __launch_bounds__(kP2PThreads)
    k_p2p(const int32_t *__restrict__ leaves, const int32_t *__restrict__ uoff,
          const int32_t *__restrict__ uidx, const int32_t *__restrict__ first,
          const int32_t *__restrict__ count, const BoxGeo *__restrict__ geo,
          const typename V4<T>::type *__restrict__ src, double D, int64_t n,
          double *__restrict__ near) {
  using V = typename V4<T>::type;
  __shared__ V ss[CAP];
  __shared__ double red[4][kP2PThreads];
  const int tid = threadIdx.x;
  const int32_t B = leaves[blockIdx.x];
  const BoxGeo gb = geo[B];
  const int32_t fb = first[B], cb = count[B];
  const int32_t e0 = uoff[B], e1 = uoff[B + 1];
  for (int32_t tc = 0; tc < cb; tc += kP2PThreads) {
    const int tcount = min(kP2PThreads, cb - tc);
    const int k = max(1, min(32, kP2PThreads / tcount));
    const int ti = tid / k, sl = tid - ti * k;
    const bool act = ti < tcount;
    V tp;
    if (act) tp = src[fb + tc + ti];
    else tp.x = tp.y = tp.z = tp.w = T(0);
    double dphi = 0, dgx = 0, dgy = 0, dgz = 0;
    int32_t e = e0, off = 0;  // next source: leaf uidx[e], point `off` within it
    while (e < e1) {
      // stage whole leaves (or pieces of an oversized one) up to CAP points
      __syncthreads();
      int nsrc = 0;
      while (e < e1) {
        const int32_t A = uidx[e];
        const int32_t ca = count[A];
        const int take = min(ca - off, CAP - nsrc);
        if (take <= 0) break;
        const BoxGeo ga = geo[A];
        const T sx = (T)center_delta(ga.ix, ga.level, gb.ix, gb.level, D);
        const T sy = (T)center_delta(ga.iy, ga.level, gb.iy, gb.level, D);
        const T sz = (T)center_delta(ga.iz, ga.level, gb.iz, gb.level, D);
        const int32_t fa = first[A] + off;
        for (int j = tid; j < take; j += kP2PThreads) {
          V v = src[fa + j];
          v.x += sx;
          v.y += sy;
          v.z += sz;
          ss[nsrc + j] = v;
        }
        nsrc += take;
        off += take;
        if (off == ca) {
          ++e;
          off = 0;
        }
      }
      __syncthreads();
      T phi = 0, gx = 0, gy = 0, gz = 0;
      if (act) {
#pragma unroll 4
        for (int j = sl; j < nsrc; j += k) {
          const V s = ss[j];
          const T dx = tp.x - s.x, dy = tp.y - s.y, dz = tp.z - s.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          const T rinv = r2 > T(0) ? rsqrt_t<T>(r2) : T(0);
          const T qr = s.w * rinv;
          const T qr3 = qr * rinv * rinv;
          phi += qr;
          gx -= qr3 * dx;
          gy -= qr3 * dy;
          gz -= qr3 * dz;
        }
      }
      dphi += (double)phi;
      dgx += (double)gx;
      dgy += (double)gy;
      dgz += (double)gz;
    }
    red[0][tid] = dphi;
    red[1][tid] = dgx;
    red[2][tid] = dgy;
    red[3][tid] = dgz;
    __syncthreads();
    if (tid < tcount) {
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      for (int s2 = 0; s2 < k; ++s2) {
        a0 += red[0][tid * k + s2];
        a1 += red[1][tid * k + s2];
        a2 += red[2][tid * k + s2];
        a3 += red[3][tid * k + s2];
      }
      const int64_t i = fb + tc + tid;
      near[i] = a0;
      near[n + i] = a1;
      near[2 * n + i] = a2;
      near[3 * n + i] = a3;
    }
    __syncthreads();
  }
}

}  // namespace

template <typename T>
void launch_p2p(int64_t nleaves, const int32_t *leaves, const int32_t *uoff, const int32_t *uidx,
                const int32_t *first, const int32_t *count, const BoxGeo *geo,
                const typename V4<T>::type *src, double D, int64_t n, double *near, cudaStream_t s) {
  if (nleaves == 0) return;
  constexpr int CAP = sizeof(T) == 4 ? 2048 : 1024;
  k_p2p<T, CAP><<<(unsigned)nleaves, kP2PThreads, 0, s>>>(leaves, uoff, uidx, first, count, geo, src,
                                                          D, n, near);
  FMM_LAUNCH_CHECK();
}

template void launch_p2p<float>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                const int32_t *, const int32_t *, const BoxGeo *, const float4 *,
                                double, int64_t, double *, cudaStream_t);
template void launch_p2p<double>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                 const int32_t *, const int32_t *, const BoxGeo *, const double4 *,
                                 double, int64_t, double *, cudaStream_t);

}  // namespace fmm

// p2p.cu -- near field: direct Green's-function interactions of each leaf's
// targets with the points of its U list (§2.2: the dense diagonal blocks of
// the hierarchical matrix are exactly the direct operator).
//
// One CTA per target leaf.  The U-list sources are staged in shared memory,
// already shifted into the target leaf's local frame (offsets between box
// centres are exact), so the inner loop is a flat sweep:
//   r2 = |x_i - x_j|^2, rinv = rsqrt(r2) (0 at r2 = 0),
//   phi += q rinv,  grad -= q rinv^3 (x_i - x_j).
// Staging reads the metadata of up to 128 source leaves at once (one thread
// each), scans their counts, and copies their points in one parallel sweep.
// Every thread owns a pair of targets (each staged source is used twice per
// load); when a leaf has fewer than 256 targets, k = floor(128 / pairs)
// threads share a pair and split its sources, and their partial sums are
// combined in FP64.  Within a staged batch each thread accumulates in T (FP32
// in mixed mode); batch totals are added in FP64.
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
  __shared__ int32_t s_incl[kP2PThreads];   // inclusive prefix of staged counts
  __shared__ int32_t s_first[kP2PThreads];  // first global point of each staged piece
  __shared__ T s_shift[3][kP2PThreads];
  __shared__ int32_t s_ws[kP2PThreads / 32];
  __shared__ double red[4][kP2PThreads];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int32_t B = leaves[blockIdx.x];
  const BoxGeo gb = geo[B];
  const int32_t fb = first[B], cb = count[B];
  const int32_t e0 = uoff[B], e1 = uoff[B + 1];
  constexpr int kChunk = 2 * kP2PThreads;  // targets per pass: two per thread
  for (int32_t tc = 0; tc < cb; tc += kChunk) {
    const int tcount = min(kChunk, cb - tc);
    const int npair = (tcount + 1) / 2;
    const int k = max(1, min(32, kP2PThreads / npair));
    const int pi = tid / k, sl = tid - pi * k;
    const bool act = pi < npair;
    const bool has1 = 2 * pi + 1 < tcount;
    V tp0, tp1;
    tp0.x = tp0.y = tp0.z = tp0.w = T(0);
    tp1 = tp0;
    if (act) tp0 = src[fb + tc + 2 * pi];
    if (act && has1) tp1 = src[fb + tc + 2 * pi + 1];
    double d0[4] = {0, 0, 0, 0}, d1[4] = {0, 0, 0, 0};
    int32_t e = e0, off = 0;  // next source: leaf uidx[e], point `off` within it
    while (e < e1) {
      __syncthreads();  // previous batch fully consumed
      // ---- metadata of up to 128 source leaves, one per thread
      int32_t c = 0, f = 0;
      T sx = T(0), sy = T(0), sz = T(0);
      if (e + tid < e1) {
        const int32_t A = uidx[e + tid];
        const BoxGeo ga = geo[A];
        const int32_t skip = tid == 0 ? off : 0;
        f = first[A] + skip;
        c = count[A] - skip;
        sx = (T)center_delta(ga.ix, ga.level, gb.ix, gb.level, D);
        sy = (T)center_delta(ga.iy, ga.level, gb.iy, gb.level, D);
        sz = (T)center_delta(ga.iz, ga.level, gb.iz, gb.level, D);
      }
      // inclusive block scan of c
      int32_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) s_ws[warp] = x;
      __syncthreads();
      int32_t base = 0;
      for (int w = 0; w < warp; ++w) base += s_ws[w];
      const int32_t incl = base + x;
      s_incl[tid] = incl;
      s_first[tid] = f;
      s_shift[0][tid] = sx;
      s_shift[1][tid] = sy;
      s_shift[2][tid] = sz;
      // leaves that fit whole (incl is non-decreasing)
      const int m = __syncthreads_count(e + tid < e1 && incl <= CAP);
      int nsrc, npiece;
      if (m == 0) {  // one oversized leaf: take CAP of its points
        nsrc = CAP;
        npiece = 1;
        off += CAP;
      } else {
        nsrc = s_incl[m - 1];
        npiece = m;
        e += m;
        off = 0;
      }
      // ---- copy the points, shifted into the target leaf's frame
      for (int idx = tid; idx < nsrc; idx += kP2PThreads) {
        int lo = 0, hi = npiece - 1;  // first piece with incl > idx
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (s_incl[mid] > idx) hi = mid;
          else lo = mid + 1;
        }
        const int32_t before = lo > 0 ? s_incl[lo - 1] : 0;
        V v = src[s_first[lo] + (idx - before)];
        v.x += s_shift[0][lo];
        v.y += s_shift[1][lo];
        v.z += s_shift[2][lo];
        ss[idx] = v;
      }
      __syncthreads();
      T a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
      if (act) {
#pragma unroll 4
        for (int j = sl; j < nsrc; j += k) {
          const V s = ss[j];
          {
            const T dx = tp0.x - s.x, dy = tp0.y - s.y, dz = tp0.z - s.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T rinv = r2 > T(0) ? rsqrt_t<T>(r2) : T(0);
            const T qr = s.w * rinv;
            const T qr3 = qr * rinv * rinv;
            a0 += qr;
            a1 -= qr3 * dx;
            a2 -= qr3 * dy;
            a3 -= qr3 * dz;
          }
          {
            const T dx = tp1.x - s.x, dy = tp1.y - s.y, dz = tp1.z - s.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            const T rinv = r2 > T(0) ? rsqrt_t<T>(r2) : T(0);
            const T qr = s.w * rinv;
            const T qr3 = qr * rinv * rinv;
            b0 += qr;
            b1 -= qr3 * dx;
            b2 -= qr3 * dy;
            b3 -= qr3 * dz;
          }
        }
      }
      d0[0] += (double)a0;
      d0[1] += (double)a1;
      d0[2] += (double)a2;
      d0[3] += (double)a3;
      d1[0] += (double)b0;
      d1[1] += (double)b1;
      d1[2] += (double)b2;
      d1[3] += (double)b3;
    }
    // combine the k partial sums of every target (two rounds: even, odd)
    for (int half = 0; half < 2; ++half) {
      const double *d = half ? d1 : d0;
      red[0][tid] = d[0];
      red[1][tid] = d[1];
      red[2][tid] = d[2];
      red[3][tid] = d[3];
      __syncthreads();
      if (tid < npair && 2 * tid + half < tcount) {
        double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
        for (int s2 = 0; s2 < k; ++s2) {
          r0 += red[0][tid * k + s2];
          r1 += red[1][tid * k + s2];
          r2 += red[2][tid * k + s2];
          r3 += red[3][tid * k + s2];
        }
        const int64_t i = fb + tc + 2 * tid + half;
        near[i] = r0;
        near[n + i] = r1;
        near[2 * n + i] = r2;
        near[3 * n + i] = r3;
      }
      __syncthreads();
    }
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

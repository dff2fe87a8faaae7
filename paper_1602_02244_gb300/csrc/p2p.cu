// p2p.cu -- near field: direct Green's-function interactions of each leaf's
// targets with the points of its U list (§2.2: the dense diagonal blocks of
// the hierarchical matrix are exactly the direct operator).
//
// One warp per target leaf, no block-wide barriers.  The warp stages its
// U-list sources in a warp-private shared buffer, already shifted into the
// target leaf's local frame (offsets between box centres are exact), and
// every lane sweeps the staged sources (broadcast shared loads) for its 1-4
// targets (the FP32 kernel splits the sources over groups of lanes when the
// leaf is small):
//   r2 = |x_i - x_j|^2, rinv = rsqrt(r2),
//   phi += q rinv,  grad -= q rinv^3 (x_i - x_j).
// Zero distances occur only between points of the same leaf (coincident
// points share a Morton key, hence a leaf), so only the leaf's own points go
// through the masked loop (rinv = 0 at r2 = 0).  Each lane accumulates a
// staged batch in T (FP32 in mixed mode) and adds batch totals in FP64.
// The FP64 kernel below is the plain form; the FP32 kernel further down packs
// the sources in pairs.
#include "eval_kernels.cuh"

namespace fmm {

namespace {

// One warp per CTA: a CTA's resources are released as soon as its leaf is
// done, so uneven leaf costs leave no idle warps holding an SM slot.
constexpr int kP2PWarps = 1;
constexpr int kP2PThreads = 32 * kP2PWarps;
constexpr int kP2PMinCtas = 16;     // resident CTAs per SM: caps registers at 128
constexpr int kP2PMinCtasF32 = 20;  // FP32 kernel (totals in shared memory): <= 102 registers
constexpr int kMaxTPL = 4;  // targets per lane

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
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
        reinterpret_cast<Dbl4 *>(near)[g] = make_dbl4(tot[t][0], tot[t][1], tot[t][2], tot[t][3]);
      }
    }
  }
}

// ---------------------------------------------------------------- FP32
// Mixed precision: the same warp-per-leaf structure, with the sources packed
// in pairs so that every FP32 instruction works on two pairs at once
// (fadd2/fmul2/ffma2).  A staged pair is two 16-byte vectors
//   (-x0, -x1, -y0, -y1) and (-z0, -z1, q0, q1)
// (negated coordinates: x_i - x_j is one packed add).  Each source leaf's
// piece is padded to an even length with a zero-charge source 1e18 away
// (finite r2, rinv ~ 1e-18, contribution exactly 0), so pairs never straddle
// pieces and only the leaf's own piece needs the zero-distance mask.  The
// gradient is accumulated as +sum q rinv^3 (x_i - x_j) and negated once.
__device__ __forceinline__ float rsqrt_approx_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

constexpr float kPadFar = 1e18f;

template <int TPL, bool kMask>
__device__ __forceinline__ void interact2(const float4 &a, const float4 &b, const float2 (&tx)[kMaxTPL],
                                          const float2 (&ty)[kMaxTPL], const float2 (&tz)[kMaxTPL],
                                          float2 (&acc)[kMaxTPL][4]) {
  const float2 nsx = make_float2(a.x, a.y), nsy = make_float2(a.z, a.w);
  const float2 nsz = make_float2(b.x, b.y), q = make_float2(b.z, b.w);
#pragma unroll
  for (int t = 0; t < TPL; ++t) {
    const float2 dx = __fadd2_rn(tx[t], nsx), dy = __fadd2_rn(ty[t], nsy), dz = __fadd2_rn(tz[t], nsz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    float2 rinv = make_float2(rsqrt_approx_ftz(r2.x), rsqrt_approx_ftz(r2.y));
    if (kMask) {
      rinv.x = r2.x > 0.f ? rinv.x : 0.f;
      rinv.y = r2.y > 0.f ? rinv.y : 0.f;
    }
    const float2 qr = __fmul2_rn(q, rinv);
    const float2 qr3 = __fmul2_rn(qr, __fmul2_rn(rinv, rinv));
    acc[t][0] = __fadd2_rn(acc[t][0], qr);
    acc[t][1] = __ffma2_rn(qr3, dx, acc[t][1]);
    acc[t][2] = __ffma2_rn(qr3, dy, acc[t][2]);
    acc[t][3] = __ffma2_rn(qr3, dz, acc[t][3]);
  }
}

// Source groups.  A leaf of c targets leaves most lanes idle in its last
// target slot when c is not near a multiple of 32 (Plummer leaves hold ~37
// points on average).  So the warp splits into G = 1, 2, 4 or 8 groups of
// 32/G lanes: a group's lanes hold the targets (1-4 each), and group g sweeps
// the staged pairs k = g (mod G).  The partial sums meet once per target tile
// (an FP64 butterfly over the groups).  G is the largest that still holds
// the leaf in one tile of 4 x 32/G targets: a second tile stages every
// source again, which costs more than the idle slots it saves (measured).
__device__ __forceinline__ int p2p_group_log2(int c) { return c <= 16 ? 3 : c <= 32 ? 2 : c <= 64 ? 1 : 0; }

// staged pairs [0, ktot) of one batch: the pairs of group gi (k = gi mod G),
// the target leaf's own piece [s0, s1) through the zero-distance mask
template <int TPL>
__device__ __forceinline__ void sweep2(const float4 *sa, const float4 *sb, int s0, int s1, int ktot, int gi,
                                       int G, const float2 (&tx)[kMaxTPL], const float2 (&ty)[kMaxTPL],
                                       const float2 (&tz)[kMaxTPL], float2 (&acc)[kMaxTPL][4]) {
#pragma unroll 2
  for (int k = gi; k < s0; k += G) interact2<TPL, false>(sa[k], sb[k], tx, ty, tz, acc);
  for (int k = s0 + ((gi - s0) & (G - 1)); k < s1; k += G) interact2<TPL, true>(sa[k], sb[k], tx, ty, tz, acc);
#pragma unroll 2
  for (int k = s1 + ((gi - s1) & (G - 1)); k < ktot; k += G) interact2<TPL, false>(sa[k], sb[k], tx, ty, tz, acc);
}

template <int CAP>
__global__ void __launch_bounds__(kP2PThreads, kP2PMinCtasF32)
    k_p2p_f32(int64_t nleaves, const int32_t *__restrict__ leaves, const int32_t *__restrict__ uoff,
              const int32_t *__restrict__ uidx, const int32_t *__restrict__ first,
              const int32_t *__restrict__ count, const BoxGeo *__restrict__ geo,
              const float4 *__restrict__ src, const double *__restrict__ side, int64_t n,
              double *__restrict__ near) {
  static_assert(CAP % 2 == 0, "pairs");
  __shared__ float4 sa_all[kP2PWarps][CAP / 2], sb_all[kP2PWarps][CAP / 2];
  __shared__ int32_t s_incl_all[kP2PWarps][32];
  // FP64 running totals of the lane's targets, [target][component][lane]:
  // touched once per staged batch, so they live in shared memory and leave
  // the registers to the inner loop (more resident warps)
  __shared__ double tot_all[kP2PWarps][kMaxTPL * 4][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t li = (int64_t)blockIdx.x * kP2PWarps + warp;
  if (li >= nleaves) return;  // whole warp: there are no block-wide barriers below
  float4 *sa = sa_all[warp], *sb = sb_all[warp];
  float *saf = reinterpret_cast<float *>(sa), *sbf = reinterpret_cast<float *>(sb);
  int32_t *s_incl = s_incl_all[warp];
  const int32_t B = leaves[li];
  const BoxGeo gb = geo[B];
  const double sbs = side[B];
  const int32_t fb = first[B], cb = count[B];
  const int32_t e0 = uoff[B], e1 = uoff[B + 1];
  const int lg = p2p_group_log2(cb);
  const int G = 1 << lg, per = 32 >> lg;
  const int gi = lane >> (5 - lg);  // this lane's source group
  const int tl = lane & (per - 1);  // its target column within the group
  for (int32_t tc = 0; tc < cb; tc += per * kMaxTPL) {
    const int tcount = min(per * kMaxTPL, cb - tc);
    const int tpl = (tcount + per - 1) / per;
    float2 tx[kMaxTPL], ty[kMaxTPL], tz[kMaxTPL];
#pragma unroll
    for (int t = 0; t < kMaxTPL; ++t) {
      const int i = tl + per * t;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < tcount) v = src[fb + tc + i];
      tx[t] = make_float2(v.x, v.x);
      ty[t] = make_float2(v.y, v.y);
      tz[t] = make_float2(v.z, v.z);
    }
    double(*tot)[32] = tot_all[warp];
#pragma unroll
    for (int q = 0; q < kMaxTPL * 4; ++q) tot[q][lane] = 0.0;
    int32_t e = e0, off = 0;  // next source: leaf uidx[e], point `off` within it
    while (e < e1) {
      // ---- metadata of up to 32 source leaves, one per lane
      int32_t c = 0, f = 0, A = -1;
      float sx = 0.f, sy = 0.f, sz = 0.f;
      if (e + lane < e1) {
        A = uidx[e + lane];
        const BoxGeo ga = geo[A];
        const int32_t skip = lane == 0 ? off : 0;
        f = first[A] + skip;
        c = count[A] - skip;
        const double sa_ = side[A];
        sx = (float)center_delta(ga.ix, sa_, gb.ix, sbs);
        sy = (float)center_delta(ga.iy, sa_, gb.iy, sbs);
        sz = (float)center_delta(ga.iz, sa_, gb.iz, sbs);
      }
      int32_t incl = c + (c & 1);  // padded to an even length
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
        const int32_t pc = __shfl_sync(0xffffffffu, c, k);
        const float px = __shfl_sync(0xffffffffu, sx, k);
        const float py = __shfl_sync(0xffffffffu, sy, k);
        const float pz = __shfl_sync(0xffffffffu, sz, k);
        const int32_t p0 = k > 0 ? s_incl[k - 1] : 0, p1 = s_incl[k];
        for (int idx = p0 + lane; idx < p1; idx += 32) {
          const int j = idx - p0;
          float nx = -kPadFar, ny = -kPadFar, nz = -kPadFar, q = 0.f;
          if (j < pc) {
            const float4 v = src[pf + j];
            nx = -(v.x + px);
            ny = -(v.y + py);
            nz = -(v.z + pz);
            q = v.w;
          }
          const int pr = idx >> 1, h = idx & 1;
          saf[4 * pr + h] = nx;
          saf[4 * pr + 2 + h] = ny;
          sbf[4 * pr + h] = nz;
          sbf[4 * pr + 2 + h] = q;
        }
      }
      __syncwarp();
      // ---- sweep the staged pairs: the pieces are contiguous and in one
      // frame, so only the target leaf's own piece (at most one) is apart
      float2 acc[kMaxTPL][4];
#pragma unroll
      for (int t = 0; t < kMaxTPL; ++t)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[t][a] = make_float2(0.f, 0.f);
      const int ktot = s_incl[npiece - 1] >> 1;
      const unsigned selfm = __ballot_sync(0xffffffffu, lane < npiece && A == B);
      int s0 = ktot, s1 = ktot;
      if (selfm) {
        const int ks = __ffs(selfm) - 1;
        s0 = (ks > 0 ? s_incl[ks - 1] : 0) >> 1;
        s1 = s_incl[ks] >> 1;
      }
      switch (tpl) {
        case 1: sweep2<1>(sa, sb, s0, s1, ktot, gi, G, tx, ty, tz, acc); break;
        case 2: sweep2<2>(sa, sb, s0, s1, ktot, gi, G, tx, ty, tz, acc); break;
        case 3: sweep2<3>(sa, sb, s0, s1, ktot, gi, G, tx, ty, tz, acc); break;
        default: sweep2<4>(sa, sb, s0, s1, ktot, gi, G, tx, ty, tz, acc); break;
      }
#pragma unroll
      for (int t = 0; t < kMaxTPL; ++t) {
        if (t >= tpl) break;
#pragma unroll
        for (int a = 0; a < 4; ++a) tot[t * 4 + a][lane] += (double)acc[t][a].x + (double)acc[t][a].y;
      }
      if (m == 0) {
        off += CAP;
      } else {
        e += m;
        off = 0;
      }
      __syncwarp();  // the staged batch is consumed before it is overwritten
    }
    // ---- the groups' partial sums of each target meet (lanes tl, tl + per, ...)
#pragma unroll
    for (int t = 0; t < kMaxTPL; ++t) {
      if (t >= tpl) break;
      double v[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) v[a] = tot[t * 4 + a][lane];
      for (int o = per; o < 32; o <<= 1)
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] += __shfl_xor_sync(0xffffffffu, v[a], o);
      const int i = tl + per * t;
      if (gi == 0 && i < tcount)
        reinterpret_cast<Dbl4 *>(near)[fb + tc + i] = make_dbl4(v[0], -v[1], -v[2], -v[3]);
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
  constexpr int CAP = sizeof(T) == 4 ? 448 : 320;  // 7 KB (FP32) / 10 KB of staged sources per warp
  if constexpr (sizeof(T) == 4) {
    // 7 KB of sources + 4 KB of FP64 totals per one-warp CTA: 20 CTAs per SM
    k_p2p_f32<CAP><<<ceil_div(nleaves, kP2PWarps), kP2PThreads, 0, s>>>(
        nleaves, leaves, uoff, uidx, first, count, geo, src, side, n, near);
  } else {
    k_p2p<T, CAP><<<ceil_div(nleaves, kP2PWarps), kP2PThreads, 0, s>>>(
        nleaves, leaves, uoff, uidx, first, count, geo, src, side, n, near);
  }
  FMM_LAUNCH_CHECK();
}

template void launch_p2p<float>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                const int32_t *, const int32_t *, const BoxGeo *, const float4 *,
                                const double *, int64_t, double *, cudaStream_t);
template void launch_p2p<double>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                 const int32_t *, const int32_t *, const BoxGeo *, const Dbl4 *,
                                 const double *, int64_t, double *, cudaStream_t);

}  // namespace fmm

// p2p.cu -- near field: direct Green's-function interactions of each leaf's
// targets with the points of its U list (§2.2: the dense diagonal blocks of
// the hierarchical matrix are exactly the direct operator).
//
// A warp per target leaf.  The warp stages its U-list sources in a
// warp-private shared buffer, in the target leaf's local frame (offsets
// between box centres are exact), and every lane sweeps the staged sources
// (broadcast shared loads) for its 1-4 targets:
//   r2 = |x_i - x_j|^2, rinv = rsqrt(r2),
//   phi += q rinv,  grad -= q rinv^3 (x_i - x_j).
// Zero distances occur only between points of the same leaf (coincident
// points share a Morton key, hence a leaf), so only the leaf's own points go
// through the masked loop (rinv = 0 at r2 = 0).
// The FP64 kernel below is the plain form (one CTA per leaf, FP64 totals per
// staged batch).  The FP32 kernel further down packs the sources in pairs,
// stages them with bulk asynchronous copies, runs persistent warps over the
// leaves in order of decreasing work class, and keeps compensated FP32 totals.
#include <algorithm>

#include "eval_kernels.cuh"
#include "tcgen05.cuh"

namespace fmm {

namespace {

// One warp per CTA: a CTA's resources are released as soon as its leaf is
// done, so uneven leaf costs leave no idle warps holding an SM slot.
constexpr int kP2PWarps = 1;
constexpr int kP2PThreads = 32 * kP2PWarps;
constexpr int kP2PMinCtas = 16;     // resident CTAs per SM: caps registers at 128
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
// (fadd2/fmul2/ffma2).  A pair is two 16-byte vectors
//   (-x0, -x1, -y0, -y1) and (-z0, -z1, q0, q1)
// (negated coordinates: x_i - x_j is one packed add).  k_p2p_pairs writes
// every leaf's points in this form once per evaluation, in the leaf's own
// frame, padded to an even count with a zero-charge source 1e18 away (finite
// r2, rinv ~ 1e-18, contribution exactly 0), so a leaf is a contiguous run of
// 32-byte pairs.  The P2P warp then moves whole leaves into shared memory
// with bulk asynchronous copies (the TMA engine, one copy per source leaf,
// completion counted in bytes on an mbarrier), two staging buffers deep: the
// copies of the next batch of U-list leaves are in flight while the current
// batch is shifted into the target leaf's frame (exact box-centre offsets,
// one rounding, as the scalar path) and swept.  The gradient is accumulated
// as +sum q rinv^3 (x_i - x_j) and negated once.
__device__ __forceinline__ float rsqrt_approx_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

constexpr float kPadFar = 1e18f;
constexpr long long kP2PWaitCycles = 400000000ll;  // ~0.2 s: far beyond any legitimate copy

// every leaf's points as pairs (see above); a warp per leaf.  The pairs of
// the leaf whose points start at `first` start at pair `first`: leaves own
// disjoint point ranges, so their ceil(count / 2) pairs never overlap (the
// buffer holds n pairs, about half of them unused).
__global__ void k_p2p_pairs(int64_t nleaves, const int32_t *__restrict__ leaves,
                            const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                            const float4 *__restrict__ src, float4 *__restrict__ pairs) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nleaves) return;
  const int32_t B = leaves[w];
  const int32_t f = first[B], c = count[B];
  const int64_t pf = f;
  const int32_t np = (c + 1) >> 1;
  for (int32_t j = lane; j < np; j += 32) {
    const float4 u = src[f + 2 * j];
    const float4 v = 2 * j + 1 < c ? src[f + 2 * j + 1] : make_float4(kPadFar, kPadFar, kPadFar, 0.f);
    pairs[2 * (pf + j)] = make_float4(-u.x, -v.x, -u.y, -v.y);
    pairs[2 * (pf + j) + 1] = make_float4(-u.z, -v.z, u.w, v.w);
  }
}

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

// staged pairs [0, ktot) of one batch (pair k at s[2k], s[2k+1]): the pairs
// of group gi (k = gi mod G), the target leaf's own piece [s0, s1) through
// the zero-distance mask
template <int TPL>
__device__ __forceinline__ void sweep2(const float4 *s, int s0, int s1, int ktot, int gi, int G,
                                       const float2 (&tx)[kMaxTPL], const float2 (&ty)[kMaxTPL],
                                       const float2 (&tz)[kMaxTPL], float2 (&acc)[kMaxTPL][4]) {
#pragma unroll 2
  for (int k = gi; k < s0; k += G) interact2<TPL, false>(s[2 * k], s[2 * k + 1], tx, ty, tz, acc);
  for (int k = s0 + ((gi - s0) & (G - 1)); k < s1; k += G)
    interact2<TPL, true>(s[2 * k], s[2 * k + 1], tx, ty, tz, acc);
#pragma unroll 2
  for (int k = s1 + ((gi - s1) & (G - 1)); k < ktot; k += G)
    interact2<TPL, false>(s[2 * k], s[2 * k + 1], tx, ty, tz, acc);
}

// Per U-list entry of the FP32 path, built once per plan (k_p2p_meta): the
// source leaf's first point and count, and the shift from its frame to the
// target leaf's, c_A - c_B.  Both centres are (anchor + 1/2) x side with
// anchors below 2^21 and power-of-two sides, so they and their difference (a
// multiple of half the smaller side, at most a side apart) are exact in FP32:
// no FP64 arithmetic, which is scarce on this GPU.  One coalesced load per
// lane gives the warp a whole batch's staging plan.
__device__ __forceinline__ float center_f32(int32_t anchor, float side) {
  return ((float)anchor + 0.5f) * side;
}

__global__ void k_p2p_meta(int64_t nleaves, const int32_t *__restrict__ leaves,
                           const int32_t *__restrict__ uoff, const int32_t *__restrict__ uidx,
                           const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                           const BoxGeo *__restrict__ geo, const double *__restrict__ side,
                           int4 *__restrict__ meta, float *__restrict__ meta_z,
                           uint64_t *__restrict__ cost_key, int32_t *__restrict__ cost_leaf) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nleaves) return;
  const int32_t B = leaves[w];
  const BoxGeo gb = geo[B];
  const float sb = (float)side[B];
  const float bx = center_f32(gb.ix, sb), by = center_f32(gb.iy, sb), bz = center_f32(gb.iz, sb);
  int32_t nsrc = 0;
  for (int32_t e = uoff[B] + lane; e < uoff[B + 1]; e += 32) {
    const int32_t A = uidx[e];
    const BoxGeo ga = geo[A];
    const float sa = (float)side[A];
    const int32_t cA = count[A];
    nsrc += cA;
    meta[e] = make_int4(first[A], cA, __float_as_int(center_f32(ga.ix, sa) - bx),
                        __float_as_int(center_f32(ga.iy, sa) - by));
    meta_z[e] = center_f32(ga.iz, sa) - bz;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nsrc += __shfl_xor_sync(0xffffffffu, nsrc, o);
  if (lane == 0) {
    // largest work first, in classes of 16x (log2(targets x sources) / 4); the
    // stable sort keeps box (Morton) order within a class, so a source leaf's
    // staged copies by neighbouring targets still meet it in L2: the same time
    // as a fine-grained order, with a fifth less DRAM traffic (measured)
    const float work = (float)count[B] * (float)nsrc + 1.0f;
    const int lv = min(65535, (int)(__log2f(work) * 0.25f));
    cost_key[w] = (uint64_t)(65535 - lv);
    cost_leaf[w] = B;
  }
}

// far + (hi + lo), the compensated near-field sum, as an FP64 value with three
// FP64 operations: Knuth's two_sum gives hi + far = s + e exactly in FP32,
// e + lo is one FP32 rounding of a term ~2^-24 below s, and the result is
// s + (e + lo) rounded once in FP64 (GB300's FP64 pipe is narrow)
__device__ __forceinline__ double add_far_near(float far, float hi, float lo) {
  const float s = __fadd_rn(hi, far);
  const float bv = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(far, bv));
  return (double)s + (double)__fadd_rn(e, lo);
}

// one staged batch: up to 32 pieces (U-list leaves, or one part of a leaf
// larger than the buffer)
struct P2PBatch {
  int ktot;    // staged pairs
  int s0, s1;  // the target leaf's own piece, if staged (else ktot, ktot)
};

// the staging plan of the 32 U entries from `e` on, one per lane
struct P2PMeta {
  int32_t first, count;  // count 0: past the end of the list
  float sx, sy, sz;
};

__device__ __forceinline__ P2PMeta p2p_load_meta(int32_t e, int32_t e1, const int4 *__restrict__ meta,
                                                 const float *__restrict__ meta_z) {
  const int lane = threadIdx.x & 31;
  P2PMeta m = {0, 0, 0.f, 0.f, 0.f};
  if (e + lane < e1) {
    const int4 v = meta[e + lane];
    m.first = v.x;
    m.count = v.y;
    m.sx = __int_as_float(v.z);
    m.sy = __int_as_float(v.w);
    m.sz = meta_z[e + lane];
  }
  return m;
}

template <int CAPP, int NBUF>
struct P2PStage {
  float4 buf[NBUF][2 * CAPP];
  uint64_t bar[NBUF];
  int32_t pend[NBUF][32];
  float shx[NBUF][32], shy[NBUF][32], shz[NBUF][32];
};

// Plans a batch from the staging plan `m` of U entries e.. (of which `off`
// pairs are already done), records its pieces in stage buffer b and issues
// its bulk copies; advances (e, off).  Warp-collective.
template <int CAPP, int NBUF>
__device__ __forceinline__ P2PBatch p2p_issue(P2PStage<CAPP, NBUF> &st, int b, const P2PMeta &m,
                                              int32_t &e, int32_t &off, int32_t fb,
                                              const float4 *__restrict__ pairs) {
  const int lane = threadIdx.x & 31;
  const int32_t skip = lane == 0 ? off : 0;
  int32_t np = m.count > 0 ? ((m.count + 1) >> 1) - skip : 0;
  const int32_t pf = m.first + skip;
  int32_t incl = np;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned fit = __ballot_sync(0xffffffffu, m.count > 0 && incl <= CAPP);
  const int mfit = __popc(fit);  // incl is non-decreasing: the first mfit leaves fit
  const int npiece = mfit == 0 ? 1 : mfit;
  if (mfit == 0) {  // one leaf larger than the buffer: CAPP of its pairs
    np = CAPP;
    incl = CAPP;
  }
  P2PBatch r;
  r.ktot = __shfl_sync(0xffffffffu, incl, npiece - 1);
  // the target leaf's own points are the only source leaf starting at fb
  const unsigned selfm = __ballot_sync(0xffffffffu, lane < npiece && m.count > 0 && m.first == fb);
  r.s0 = r.s1 = r.ktot;
  if (selfm) {
    const int ks = __ffs(selfm) - 1;
    r.s0 = __shfl_sync(0xffffffffu, incl - np, ks);
    r.s1 = __shfl_sync(0xffffffffu, incl, ks);
  }
  if (lane < npiece) {
    st.pend[b][lane] = incl;
    st.shx[b][lane] = m.sx;
    st.shy[b][lane] = m.sy;
    st.shz[b][lane] = m.sz;
  }
  // the buffer's previous contents were read (and written) through the
  // generic proxy; order those accesses before the async-proxy copies
  tc::fence_async_shared();
  __syncwarp();
  if (lane == 0) tc::mbar_arrive_expect_tx(&st.bar[b], (uint32_t)r.ktot * 32u);
  if (lane < npiece && np > 0)
    tc::bulk_g2s(&st.buf[b][2 * (incl - np)], pairs + 2 * (int64_t)pf, (uint32_t)np * 32u, &st.bar[b]);
  if (mfit == 0) {
    off += CAPP;
  } else {
    e += mfit;
    off = 0;
  }
  return r;
}

// NBUF = 2: the copies of batch k+1 are in flight while batch k is swept;
// NBUF = 1: one buffer, refilled after each sweep.  The staging plan of the
// batch after the next is loaded one batch ahead in either case.
// Persistent: one warp per CTA, as many CTAs as fit on the GPU at once; each
// takes leaves from `order` (most work first) through an atomic ticket, the
// next ticket fetched while the current leaf runs, so no SM idles on CTA
// launches and the last leaves to start are the cheapest.
template <int CAPP, int NBUF, int MINB>
__global__ void __launch_bounds__(kP2PThreads, MINB)
    k_p2p_f32(int64_t nleaves, const int32_t *__restrict__ order, const int32_t *__restrict__ uoff,
              const int4 *__restrict__ meta, const float *__restrict__ meta_z,
              const int32_t *__restrict__ first, const int32_t *__restrict__ count,
              const float4 *__restrict__ src, const float4 *__restrict__ pairs,
              const float4 *__restrict__ far, const int32_t *__restrict__ perm,
              double *__restrict__ phi, double *__restrict__ grad, int *__restrict__ ticket,
              int *__restrict__ err) {
  static_assert(kP2PWarps == 1, "one warp per CTA: the staging buffers are the CTA's");
  __shared__ __align__(16) P2PStage<CAPP, NBUF> st;
  // Compensated running totals of the lane's targets, [target][component][lane]
  // = (sum, error term), both FP32: each staged batch's FP32 sum is added by
  // an error-free transformation (two_sum), so the total carries about twice
  // FP32's precision without FP64 arithmetic, which runs at a small fraction
  // of the FP32 rate on this GPU.  Touched once per batch, the totals live in
  // shared memory and leave the registers to the inner loop.
  __shared__ float2 tot[kMaxTPL * 4][32];
  const int lane = threadIdx.x & 31;
  if (lane == 0)
    for (int q = 0; q < NBUF; ++q) tc::mbar_init(&st.bar[q], 1);
  __syncwarp();
  uint32_t phase = 0;    // bit b: parity of the next phase of st.bar[b]
  unsigned pending = 0;  // bit b: copies issued into buffer b and not yet waited for
  bool failed = false;
  int li = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(ticket, 1) : 0, 0);
  while (li < nleaves && !failed) {
    const int next_li = lane == 0 ? atomicAdd(ticket, 1) : 0;  // used after this leaf
    const int32_t B = order[li];
    const int32_t fb = first[B], cb = count[B];
    const int32_t e0 = uoff[B], e1 = uoff[B + 1];
    const int lg = p2p_group_log2(cb);
    const int G = 1 << lg, per = 32 >> lg;
    const int gi = lane >> (5 - lg);  // this lane's source group
    const int tl = lane & (per - 1);  // its target column within the group
    for (int32_t tc = 0; tc < cb && !failed; tc += per * kMaxTPL) {
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
  #pragma unroll
      for (int q = 0; q < kMaxTPL * 4; ++q) tot[q][lane] = make_float2(0.f, 0.f);
      int32_t e = e0, off = 0;  // next source: U entry e, pair `off` within it
      int b = 0;
      P2PBatch cur = {0, 0, 0};
      P2PMeta m = p2p_load_meta(e, e1, meta, meta_z);
      bool have = e < e1;
      if (have) {
        cur = p2p_issue<CAPP, NBUF>(st, b, m, e, off, fb, pairs);
        pending |= 1u << b;
        m = p2p_load_meta(e, e1, meta, meta_z);
      }
      while (have) {
        P2PBatch nxt = {0, 0, 0};
        bool more = e < e1;
        if (NBUF == 2 && more) {  // the next batch's copies go out before this one is waited for
          nxt = p2p_issue<CAPP, NBUF>(st, b ^ 1, m, e, off, fb, pairs);
          pending |= 1u << (b ^ 1);
          m = p2p_load_meta(e, e1, meta, meta_z);
        }
        const bool ok = tc::mbar_wait_bounded(&st.bar[b], (phase >> b) & 1u, kP2PWaitCycles);
        if (!__all_sync(0xffffffffu, ok)) {
          failed = true;
          break;
        }
        phase ^= 1u << b;
        pending &= ~(1u << b);
        // ---- shift the batch into the target leaf's frame, in place
        float4 *sbuf = st.buf[b];
        int k = 0;
        for (int idx = lane; idx < cur.ktot; idx += 32) {
          while (st.pend[b][k] <= idx) ++k;
          const float sx = st.shx[b][k], sy = st.shy[b][k], sz = st.shz[b][k];
          float4 a = sbuf[2 * idx], c = sbuf[2 * idx + 1];
          a.x -= sx;
          a.y -= sx;
          a.z -= sy;
          a.w -= sy;
          c.x -= sz;
          c.y -= sz;
          sbuf[2 * idx] = a;
          sbuf[2 * idx + 1] = c;
        }
        __syncwarp();
        // ---- sweep the staged pairs: the pieces are contiguous and in one
        // frame, so only the target leaf's own piece (at most one) is apart
        float2 acc[kMaxTPL][4];
  #pragma unroll
        for (int t = 0; t < kMaxTPL; ++t)
  #pragma unroll
          for (int a = 0; a < 4; ++a) acc[t][a] = make_float2(0.f, 0.f);
        switch (tpl) {
          case 1: sweep2<1>(sbuf, cur.s0, cur.s1, cur.ktot, gi, G, tx, ty, tz, acc); break;
          case 2: sweep2<2>(sbuf, cur.s0, cur.s1, cur.ktot, gi, G, tx, ty, tz, acc); break;
          case 3: sweep2<3>(sbuf, cur.s0, cur.s1, cur.ktot, gi, G, tx, ty, tz, acc); break;
          default: sweep2<4>(sbuf, cur.s0, cur.s1, cur.ktot, gi, G, tx, ty, tz, acc); break;
        }
  #pragma unroll
        for (int t = 0; t < kMaxTPL; ++t) {
          if (t >= tpl) break;
  #pragma unroll
          for (int a = 0; a < 4; ++a) {
            float2 &T = tot[t * 4 + a][lane];
            const float v = __fadd_rn(acc[t][a].x, acc[t][a].y);
            // two_sum: s + err == T.x + v exactly (Knuth)
            const float sum = __fadd_rn(T.x, v);
            const float bv = __fsub_rn(sum, T.x);
            const float err = __fadd_rn(__fsub_rn(T.x, __fsub_rn(sum, bv)), __fsub_rn(v, bv));
            T = make_float2(sum, __fadd_rn(T.y, err));
          }
        }
        __syncwarp();  // buffer b is consumed before a batch refills it
        if (NBUF == 1 && more) {
          nxt = p2p_issue<CAPP, NBUF>(st, b, m, e, off, fb, pairs);
          pending |= 1u << b;
          m = p2p_load_meta(e, e1, meta, meta_z);
        }
        cur = nxt;
        have = more;
        if (NBUF == 2) b ^= 1;
      }
      if (failed) break;
      // ---- the groups' partial sums of each target meet (lanes tl, tl + per,
      // ...), still as compensated FP32 pairs; FP64 only for the stored sums
  #pragma unroll
      for (int t = 0; t < kMaxTPL; ++t) {
        if (t >= tpl) break;
        float h[4], l[4];
  #pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 T = tot[t * 4 + a][lane];
          h[a] = T.x;
          l[a] = T.y;
        }
        for (int o = per; o < 32; o <<= 1)
  #pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h[a], o);
            const float l2 = __shfl_xor_sync(0xffffffffu, l[a], o);
            const float sum = __fadd_rn(h[a], h2);
            const float bv = __fsub_rn(sum, h[a]);
            const float err = __fadd_rn(__fsub_rn(h[a], __fsub_rn(sum, bv)), __fsub_rn(h2, bv));
            h[a] = sum;
            l[a] = __fadd_rn(__fadd_rn(l[a], l2), err);
          }
        // the target is finished here: far field + near field, written at its
        // input index (the gradient of 1/r points away from the sources)
        const int i = tl + per * t;
        if (gi == 0 && i < tcount) {
          const int64_t si = fb + tc + i;
          const float4 fr = far[si];
          const int64_t o = perm[si];
          phi[o] = add_far_near(fr.x, h[0], l[0]);
          if (grad) {
            grad[3 * o] = add_far_near(fr.y, -h[1], -l[1]);
            grad[3 * o + 1] = add_far_near(fr.z, -h[2], -l[2]);
            grad[3 * o + 2] = add_far_near(fr.w, -h[3], -l[3]);
          }
        }
      }
    }
    li = __shfl_sync(0xffffffffu, next_li, 0);
  }
  if (failed) {
    // copies still in flight land before the CTA's shared memory is released
    if (lane == 0) atomicExch(err, 1);
    for (int bb = 0; bb < NBUF; ++bb)
      if (pending & (1u << bb)) tc::mbar_wait_bounded(&st.bar[bb], (phase >> bb) & 1u, kP2PWaitCycles);
  }
}

// FP32 staging shapes (the `p2p_tile` option; the autotuner picks one):
// pairs per buffer, buffers, and the resident CTAs the registers are held to
struct P2PTile {
  int capp, nbuf, minb;
};
constexpr P2PTile kP2PTiles[] = {{160, 2, 16}, {96, 2, 20}, {224, 1, 20}, {128, 1, 24}};

}  // namespace

void launch_p2p_meta(int64_t nleaves, const int32_t *leaves, const int32_t *uoff, const int32_t *uidx,
                     const int32_t *first, const int32_t *count, const BoxGeo *geo, const double *side,
                     int4 *meta, float *meta_z, uint64_t *cost_key, int32_t *cost_leaf, cudaStream_t s) {
  if (nleaves == 0) return;
  constexpr int kLeafWarps = 8;
  k_p2p_meta<<<ceil_div(nleaves, kLeafWarps), 32 * kLeafWarps, 0, s>>>(
      nleaves, leaves, uoff, uidx, first, count, geo, side, meta, meta_z, cost_key, cost_leaf);
  FMM_LAUNCH_CHECK();
}

namespace {
// resident CTAs of a persistent kernel on the current device
template <typename K>
int persistent_grid(K kern, int64_t work) {
  static int per_sm = 0;  // the same for every device of this kind
  if (per_sm == 0) {
    int v = 0;
    FMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kP2PThreads, 0));
    per_sm = v > 0 ? v : 1;
  }
  int dev = 0, sms = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  FMM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return (int)std::min<int64_t>(work, (int64_t)sms * per_sm);
}
}  // namespace

template <typename T>
void launch_p2p(int64_t nleaves, const int32_t *leaves, const int32_t *uoff, const int32_t *uidx,
                const int32_t *first, const int32_t *count, const BoxGeo *geo,
                const typename V4<T>::type *src, const double *side, int64_t n, double *near,
                P2PScratch *scratch, cudaStream_t s) {
  if (nleaves == 0) return;
  if constexpr (sizeof(T) == 4) {
    constexpr int kLeafWarps = 8;
    k_p2p_pairs<<<ceil_div(nleaves, kLeafWarps), 32 * kLeafWarps, 0, s>>>(
        nleaves, leaves, first, count, src, scratch->pairs);
    FMM_LAUNCH_CHECK();
    FMM_CUDA(cudaMemsetAsync(scratch->ticket, 0, sizeof(int), s));
    auto run = [&](auto kern) {
      kern<<<persistent_grid(kern, nleaves), kP2PThreads, 0, s>>>(
          nleaves, scratch->order, uoff, scratch->meta, scratch->meta_z, first, count, src,
          scratch->pairs, scratch->far, scratch->perm, scratch->phi, scratch->grad, scratch->ticket,
          scratch->err);
    };
    switch (scratch->tile) {
      case 1: run(k_p2p_f32<kP2PTiles[0].capp, kP2PTiles[0].nbuf, kP2PTiles[0].minb>); break;
      case 2: run(k_p2p_f32<kP2PTiles[1].capp, kP2PTiles[1].nbuf, kP2PTiles[1].minb>); break;
      case 3: run(k_p2p_f32<kP2PTiles[2].capp, kP2PTiles[2].nbuf, kP2PTiles[2].minb>); break;
      default: run(k_p2p_f32<kP2PTiles[3].capp, kP2PTiles[3].nbuf, kP2PTiles[3].minb>); break;
    }
  } else {
    constexpr int CAP = 320;  // 10 KB of staged sources per warp
    k_p2p<T, CAP><<<ceil_div(nleaves, kP2PWarps), kP2PThreads, 0, s>>>(
        nleaves, leaves, uoff, uidx, first, count, geo, src, side, n, near);
  }
  FMM_LAUNCH_CHECK();
}

int p2p_num_tiles() { return (int)(sizeof(kP2PTiles) / sizeof(kP2PTiles[0])); }

size_t p2p_pair_floats(int64_t n) { return 8 * (size_t)(n + 1); }

template void launch_p2p<float>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                const int32_t *, const int32_t *, const BoxGeo *, const float4 *,
                                const double *, int64_t, double *, P2PScratch *, cudaStream_t);
template void launch_p2p<double>(int64_t, const int32_t *, const int32_t *, const int32_t *,
                                 const int32_t *, const int32_t *, const BoxGeo *, const Dbl4 *,
                                 const double *, int64_t, double *, P2PScratch *, cudaStream_t);

}  // namespace fmm

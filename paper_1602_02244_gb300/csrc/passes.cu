// passes.cu -- the upward and downward passes of the FMM mat-vec (§1: the
// analytic FMM as a matrix-free H^2 mat-vec; translation operators of §2.2):
// P2M at leaves, M2M child -> parent, P2L over X lists, L2L parent -> child,
// L2P at leaf targets, M2P over W lists, and the per-target reduction.
//
// Coefficients are scale-free and stored in the real basis described in
// operators.cu.  Point data are leaf-local: (x - c_leaf, y - c_leaf,
// z - c_leaf, q); box-to-box centre offsets come exactly from integer anchors.
#include "eval_kernels.cuh"
#include "harmonics.cuh"

#include <type_traits>

namespace fmm {

namespace {

__device__ __forceinline__ double center_delta(int32_t ia, double sa, int32_t ib, double sb) {
  // (c_A - c_B) along one axis from anchors and box sides, exact: both centres
  // are dyadic multiples of the root side
  return ((double)ia + 0.5) * sa - ((double)ib + 0.5) * sb;
}

constexpr int kAccSlots = 14;  // ceil(441 / 32): coefficients per lane for p <= 20

// Per-lane coefficient sums fit in registers (at most 128 32-bit words) when
// the order is a compile-time constant.
template <typename T, int PT>
constexpr bool reg_accumulate() {
  return PT > 0 && ncoef(PT) * (int)sizeof(T) <= 4 * 128;
}


// Warp reduction of NC per-lane sums through a shared-memory transpose: every
// lane writes its column of buf (NC x 33), then lane l adds up rows l, l + 32,
// ... over the 32 columns.  ~3 NC instructions per lane instead of the ~10 NC
// of a shuffle tree.  ADD: add into row[k]; else store and zero the padding
// up to ld (and mirror into row64 when given).
template <bool ADD, typename T, int NC>
__device__ __forceinline__ void transpose_sums(const T (&racc)[NC], int lane, T *buf, T *row, int ld,
                                               double *row64) {
#pragma unroll
  for (int k = 0; k < NC; ++k) buf[k * 33 + lane] = racc[k];
  __syncwarp();
  for (int k = lane; k < NC; k += 32) {
    T v = T(0);
#pragma unroll 8
    for (int j = 0; j < 32; ++j) v += buf[k * 33 + j];
    if (ADD) {
      row[k] += v;
    } else {
      row[k] = v;
      if (row64) row64[k] = (double)v;
    }
  }
  if (!ADD)
    for (int k = NC + lane; k < ld; k += 32) {
      row[k] = T(0);
      if (row64) row64[k] = 0.0;
    }
  __syncwarp();
}


template <typename T>
__global__ void k_permute_charges(int64_t n, const int32_t *__restrict__ perm,
                                  const double *__restrict__ q, const typename V4<T>::type *pl,
                                  typename V4<T>::type *__restrict__ src) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  typename V4<T>::type v = pl[i];
  v.w = (T)q[perm[i]];
  src[i] = v;
}

// P2M: M^_n^m = sum_j q_j conj(R_n^m((x_j - c)/a)); one warp per leaf, lanes
// over points, a warp-private shared buffer transposes per-point harmonics
// into per-coefficient sums.
template <typename T, int PT>
__global__ void k_p2m(int p_rt, int64_t nleaves, const int32_t *__restrict__ leaves,
                      const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                      const BoxGeo *__restrict__ geo, const typename V4<T>::type *__restrict__ src,
                      const double *__restrict__ side, T *__restrict__ M, double *__restrict__ M64,
                      int coarse) {
  const int p = PT > 0 ? PT : p_rt;  // compile-time order unrolls the harmonic streams
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = ncoef(p), ld = coef_pitch(p), pitch = 33, lane = threadIdx.x & 31;
  T *buf = reinterpret_cast<T *>(smem_raw) + (size_t)(threadIdx.x >> 5) * nc * pitch;
  int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nleaves) return;
  const int32_t b = leaves[w];
  const BoxGeo g = geo[b];
  const T inva = (T)(1.0 / side[b]);
  if constexpr (reg_accumulate<T, PT>()) {  // per-lane sums in registers, one warp reduction
    constexpr int NC = ncoef(PT);
    T racc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) racc[k] = T(0);
    const int32_t f = first[b], c = count[b];
    for (int32_t j = lane; j < c; j += 32) {
      const typename V4<T>::type s = src[f + j];
      const T q = s.w;
      regular_stream<T>(PT, s.x * inva, s.y * inva, s.z * inva, [&](int n, int m, T re, T im) {
        racc[cidx(n, m)] += q * re;
        if (m > 0) racc[cidx(n, -m)] -= q * im;
      });
    }
    transpose_sums<false, T, NC>(racc, lane, buf, M + (int64_t)b * ld, ld,
                                 (M64 && g.level <= coarse) ? M64 + (int64_t)b * ld : nullptr);
  } else {  // run-time order: per-point columns summed in shared memory
    T acc[kAccSlots];
#pragma unroll
    for (int t = 0; t < kAccSlots; ++t) acc[t] = T(0);
    const int32_t f = first[b], c = count[b];
    for (int32_t j0 = 0; j0 < c; j0 += 32) {
      const int32_t j = j0 + lane;
      if (j < c) {
        const typename V4<T>::type s = src[f + j];
        const T q = s.w;
        regular_stream<T>(p, s.x * inva, s.y * inva, s.z * inva, [&](int n, int m, T re, T im) {
          buf[cidx(n, m) * pitch + lane] = q * re;
          if (m > 0) buf[cidx(n, -m) * pitch + lane] = -q * im;
        });
      } else {
        for (int k = 0; k < nc; ++k) buf[k * pitch + lane] = T(0);
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kAccSlots; ++t) {
        const int k = lane + 32 * t;
        if (k < nc) {
          T s = T(0);
          for (int jj = 0; jj < 32; ++jj) s += buf[k * pitch + jj];
          acc[t] += s;
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < kAccSlots; ++t) {  // the row padding is written as zero
      const int k = lane + 32 * t;
      if (k < ld) {
        M[(int64_t)b * ld + k] = acc[t];
        if (M64 && g.level <= coarse) M64[(int64_t)b * ld + k] = (double)acc[t];
      }
    }
  }
}

// P2L over X lists: L^_n^m(C) += sum_{A in X(C)} sum_{j in A} q_j conj(I_n^m((x_j - c_C)/a_C))
template <typename T, int PT>
__global__ void k_p2l(int p_rt, int64_t nboxes_x, const int32_t *__restrict__ xboxes,
                      const int32_t *__restrict__ xoff, const int32_t *__restrict__ xidx,
                      const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                      const BoxGeo *__restrict__ geo, const typename V4<T>::type *__restrict__ src,
                      const double *__restrict__ side, T *__restrict__ L) {
  const int p = PT > 0 ? PT : p_rt;  // compile-time order unrolls the harmonic streams
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = ncoef(p), ld = coef_pitch(p), pitch = 33, lane = threadIdx.x & 31;
  T *buf = reinterpret_cast<T *>(smem_raw) + (size_t)(threadIdx.x >> 5) * nc * pitch;
  int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= nboxes_x) return;
  const int32_t C = xboxes[w];
  const BoxGeo gc = geo[C];
  const double ac = side[C];
  const T inva = (T)(1.0 / ac);
  if constexpr (reg_accumulate<T, PT>()) {  // per-lane sums in registers, one warp reduction
    constexpr int NC = ncoef(PT);
    T racc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) racc[k] = T(0);
    // The X list's source points are taken as one concatenated range, 32 at
    // a time, so small source leaves do not leave lanes idle: up to 32 leaves'
    // metadata sit one per lane, and a lane finds the leaf of its point by a
    // binary search over the inclusive counts (shuffles).
    const int32_t x1 = xoff[C + 1];
    for (int32_t eb = xoff[C]; eb < x1; eb += 32) {
      int32_t c = 0, f = 0;
      T sx = T(0), sy = T(0), sz = T(0);
      if (eb + lane < x1) {
        const int32_t A = xidx[eb + lane];
        const BoxGeo ga = geo[A];
        c = count[A];
        f = first[A];
        sx = (T)center_delta(ga.ix, side[A], gc.ix, ac);
        sy = (T)center_delta(ga.iy, side[A], gc.iy, ac);
        sz = (T)center_delta(ga.iz, side[A], gc.iz, ac);
      }
      int32_t incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
      const int32_t excl = incl - c;
      for (int32_t base = 0; base < total; base += 32) {  // warp-uniform trip count
        const int32_t idx = base + lane;
        int k = 0;  // first leaf whose inclusive count exceeds idx
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int32_t v = __shfl_sync(0xffffffffu, incl, k + step - 1);
          if (v <= idx) k += step;
        }
        const int32_t fk = __shfl_sync(0xffffffffu, f, k), ek = __shfl_sync(0xffffffffu, excl, k);
        const T ox = __shfl_sync(0xffffffffu, sx, k), oy = __shfl_sync(0xffffffffu, sy, k),
                oz = __shfl_sync(0xffffffffu, sz, k);
        if (idx < total) {
          const typename V4<T>::type sp = src[fk + (idx - ek)];
          const T q = sp.w;
          irregular_stream<T>(PT, (sp.x + ox) * inva, (sp.y + oy) * inva, (sp.z + oz) * inva,
                              [&](int n, int m, T re, T im) {
                                racc[cidx(n, m)] += q * re;
                                if (m > 0) racc[cidx(n, -m)] -= q * im;
                              });
        }
      }
    }
    transpose_sums<true, T, NC>(racc, lane, buf, L + (int64_t)C * ld, ld, nullptr);
  } else {  // run-time order: per-point columns summed in shared memory
    T acc[kAccSlots];
#pragma unroll
    for (int t = 0; t < kAccSlots; ++t) acc[t] = T(0);
    for (int32_t e = xoff[C]; e < xoff[C + 1]; ++e) {
      const int32_t A = xidx[e];
      const BoxGeo ga = geo[A];
      const T sx = (T)center_delta(ga.ix, side[A], gc.ix, ac);
      const T sy = (T)center_delta(ga.iy, side[A], gc.iy, ac);
      const T sz = (T)center_delta(ga.iz, side[A], gc.iz, ac);
      const int32_t f = first[A], c = count[A];
      for (int32_t j0 = 0; j0 < c; j0 += 32) {
        const int32_t j = j0 + lane;
        if (j < c) {
          const typename V4<T>::type s = src[f + j];
          const T q = s.w;
          irregular_stream<T>(p, (s.x + sx) * inva, (s.y + sy) * inva, (s.z + sz) * inva,
                              [&](int n, int m, T re, T im) {
                                buf[cidx(n, m) * pitch + lane] = q * re;
                                if (m > 0) buf[cidx(n, -m) * pitch + lane] = -q * im;
                              });
        } else {
          for (int k = 0; k < nc; ++k) buf[k * pitch + lane] = T(0);
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kAccSlots; ++t) {
          const int k = lane + 32 * t;
          if (k < nc) {
            T s = T(0);
            for (int jj = 0; jj < 32; ++jj) s += buf[k * pitch + jj];
            acc[t] += s;
          }
        }
        __syncwarp();
      }
    }
#pragma unroll
    for (int t = 0; t < kAccSlots; ++t) {
      const int k = lane + 32 * t;
      if (k < nc) L[(int64_t)C * ld + k] += acc[t];
    }
  }
}

__device__ __forceinline__ int degree_of(int r) {
  int n = (int)sqrtf((float)r);
  while (n * n > r) --n;
  while ((n + 1) * (n + 1) <= r) ++n;
  return n;
}

__device__ __forceinline__ int octant(const BoxGeo &g) {
  return (g.ix & 1) | ((g.iy & 1) << 1) | ((g.iz & 1) << 2);
}

// M2M into the parents of one level: thread per (parent, output coefficient);
// output degree n uses inputs of degree <= n only.
template <typename Tin, typename Tout, typename Top, typename Tacc>
__global__ void k_m2m(int p, int32_t b0, int32_t nbl, const int32_t *__restrict__ child,
                      const int32_t *__restrict__ nchild, const BoxGeo *__restrict__ geo,
                      const Tin *__restrict__ Mc, const Top *__restrict__ ops, Tout *__restrict__ Mp,
                      float *__restrict__ Mp32) {
  // 8 consecutive lanes per (parent, output): lane c takes the c-th child
  // and a 3-step shuffle reduction sums them (short dependent chains)
  const int nc = ncoef(p), ld = coef_pitch(p);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = t >> 3;
  const int c = (int)(t & 7);
  const bool in = g < (int64_t)nbl * ld;
  int32_t b = 0, nch = 0;
  int r = 0;
  if (in) {
    b = b0 + (int32_t)(g / ld);
    r = (int)(g % ld);
    nch = nchild[b];
  }
  Tacc acc = Tacc(0);
  if (in && r < nc && c < nch) {  // the row padding is written as zero
    const int kmax = ncoef(degree_of(r));
    const int32_t cc = child[b] + c;
    const Top *row = ops + ((size_t)octant(geo[cc]) * nc + r) * nc;
    const Tin *m = Mc + (int64_t)cc * ld;
    for (int k = 0; k < kmax; ++k) acc += (Tacc)row[k] * (Tacc)m[k];
  }
#pragma unroll
  for (int o = 1; o < 8; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (!in || c != 0 || nch == 0) return;  // a leaf keeps its P2M multipole
  Mp[(int64_t)b * ld + r] = (Tout)acc;
  if (Mp32) Mp32[(int64_t)b * ld + r] = (float)acc;
}

// L2L into the boxes of one level: L(child) = L_self(child) + T(octant) L(parent);
// output degree n uses inputs of degree >= n only.
template <typename Tself, typename Tpar, typename Tout, typename Top, typename Tacc>
__global__ void k_l2l(int p, int32_t b0, int32_t nbl, const int32_t *__restrict__ parent,
                      const BoxGeo *__restrict__ geo, const Tself *Lself, const Tpar *Lpar,
                      const Top *__restrict__ ops, Tout *Lout, float *Lout32) {
  const int nc = ncoef(p), ld = coef_pitch(p);
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nbl * nc) return;
  const int32_t b = b0 + (int32_t)(t / nc);
  const int r = (int)(t % nc);
  const int32_t P = parent[b];
  const int n = degree_of(r);
  const Top *row = ops + ((size_t)octant(geo[b]) * nc + r) * nc;
  const Tpar *lp = Lpar + (int64_t)P * ld;
  Tacc acc = (Tacc)Lself[(int64_t)b * ld + r];
  for (int k = n * n; k < nc; ++k) acc += (Tacc)row[k] * (Tacc)lp[k];
  Lout[(int64_t)b * ld + r] = (Tout)acc;
  if (Lout32) Lout32[(int64_t)b * ld + r] = (float)acc;
}

// FP32 M2M and L2L as small GEMMs per child octant.  The boxes of a level
// are grouped by their octant within the parent (plan time), so a CTA takes
// up to kTrRows boxes of one level and one octant, all translated by the same
// operator: the input-major operator opT[o] ((p+1)^2 x coef_pitch(p) floats)
// and the tile's input rows (k-major) are staged in shared memory, and each
// thread accumulates one output quad (4 coefficients) of 8 rows in
// registers -- per input coefficient one 16-byte operator load (different per
// quad, conflict-free) and two broadcast 16-byte loads of the 8 inputs serve
// 32 multiply-adds.  The triangular structure bounds the loops: M2M output
// degree n uses inputs of degree <= n, L2L inputs of degree >= n.
//   M2M: part[child] = opT[o]^T M[child], then each parent sums its children's
//        parts in child order (deterministic);
//   L2L: L[child] += opT[o]^T L[parent of child].
// Each output sums its inputs from the highest degree down, smaller terms
// first: in FP32 that order gives the lower rounding error (measured on the
// 4M Plummer case: 4.87e-7 against 5.40e-7 in ascending order).
constexpr int kTrRows = 64;              // boxes per CTA
constexpr int kL2LLanesMaxBoxes = 12000;  // smaller L2L levels take k_l2l_lanes
constexpr int kTrPitch = kTrRows + 4;    // shared input row: 16-byte aligned, fewer conflicts
constexpr int kMaxLevels = 32;
struct LevelOffsets {
  int32_t off[kMaxLevels + 1];
  int n;  // levels
};

__device__ __forceinline__ int level_of(const LevelOffsets &lo, int32_t b) {
  int l = 0;
  while (l + 1 < lo.n && lo.off[l + 1] <= b) ++l;
  return l;
}

__global__ void k_oct_count(int32_t b0, int32_t nb, LevelOffsets lo, const BoxGeo *__restrict__ geo,
                            int32_t *__restrict__ cnt, int32_t *__restrict__ pos) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= nb) return;
  const int32_t b = b0 + i;
  pos[i] = atomicAdd(&cnt[level_of(lo, b) * 9 + octant(geo[b])], 1);
}

__global__ void k_oct_scan(LevelOffsets lo, int32_t *__restrict__ off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int l = 0; l < lo.n; ++l) {
    int32_t run = lo.off[l];
    for (int o = 0; o < 8; ++o) {
      const int32_t c = off[l * 9 + o];
      off[l * 9 + o] = run;
      run += c;
    }
    off[l * 9 + 8] = lo.off[l + 1];
  }
}

__global__ void k_oct_scatter(int32_t b0, int32_t nb, LevelOffsets lo, const BoxGeo *__restrict__ geo,
                              const int32_t *__restrict__ off, const int32_t *__restrict__ pos,
                              int32_t *__restrict__ order) {
  const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= nb) return;
  const int32_t b = b0 + i;
  order[off[level_of(lo, b) * 9 + octant(geo[b])] + pos[i]] = b;
}

template <bool L2L>
__global__ void k_trans_oct(int p, int l, const int32_t *__restrict__ oct_off,
                            const int32_t *__restrict__ oct_order, const int32_t *__restrict__ parent,
                            const float4 *__restrict__ opT, const float *in, float *out) {
  extern __shared__ __align__(16) float tr_sm[];
  __shared__ int32_t s_off[9], s_src[kTrRows], s_dst[kTrRows];
  const int nc = ncoef(p), ld = coef_pitch(p), nq = ld / 4;
  float *B = tr_sm;                    // [nc][ld]: opT[o]
  float *A = tr_sm + (size_t)nc * ld;  // [nc][kTrPitch]: input k of row j at A[k][j]
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid < 9) s_off[tid] = oct_off[l * 9 + tid];
  __syncthreads();
  // this CTA's octant and tile (the same in every thread)
  int o = 0, t = (int)blockIdx.x;
  for (; o < 8; ++o) {
    const int nt = (s_off[o + 1] - s_off[o] + kTrRows - 1) / kTrRows;
    if (t < nt) break;
    t -= nt;
  }
  if (o == 8) return;
  const int32_t r0 = s_off[o] + t * kTrRows;
  const int nr = min(kTrRows, s_off[o + 1] - r0);
  for (int j = tid; j < nr; j += nthr) {
    const int32_t box = oct_order[r0 + j];
    s_dst[j] = box;
    s_src[j] = L2L ? parent[box] : box;
  }
  const float4 *src = opT + (size_t)o * nc * nq;
  for (int i = tid; i < nc * nq; i += nthr) reinterpret_cast<float4 *>(B)[i] = src[i];
  __syncthreads();
  for (int i = tid; i < kTrRows * nc; i += nthr) {
    const int j = i / nc, k = i - j * nc;
    A[k * kTrPitch + j] = j < nr ? in[(int64_t)s_src[j] * ld + k] : 0.f;
  }
  __syncthreads();
  // compute role: output quad q of rows 8 g .. 8 g + 7
  if (tid >= 8 * nq) return;
  const int q = tid % nq, g = tid / nq;
  if (8 * g >= nr) return;
  const int dq = degree_of(min(4 * q + 3, nc - 1)), d0 = degree_of(4 * q);
  const int k0 = L2L ? d0 * d0 : 0, k1 = L2L ? nc : (dq + 1) * (dq + 1);
  float4 acc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = k1 - 1; k >= k0; --k) {  // high degrees first: the smaller terms
    const float4 w = reinterpret_cast<const float4 *>(B + (size_t)k * ld)[q];
    const float4 a0 = reinterpret_cast<const float4 *>(A + (size_t)k * kTrPitch)[2 * g];
    const float4 a1 = reinterpret_cast<const float4 *>(A + (size_t)k * kTrPitch)[2 * g + 1];
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      acc[i].x = fmaf(w.x, a[i], acc[i].x);
      acc[i].y = fmaf(w.y, a[i], acc[i].y);
      acc[i].z = fmaf(w.z, a[i], acc[i].z);
      acc[i].w = fmaf(w.w, a[i], acc[i].w);
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = 8 * g + i;
    if (j >= nr) break;
    float4 *dst = reinterpret_cast<float4 *>(out + (int64_t)s_dst[j] * ld) + q;
    if (L2L) {
      float4 v = *dst;
      v.x += acc[i].x;
      v.y += acc[i].y;
      v.z += acc[i].z;
      v.w += acc[i].w;
      *dst = v;
    } else {
      *dst = acc[i];
    }
  }
}

// FP32 L2L for small levels (a few thousand boxes), where the per-octant tiles
// below are bound by one CTA's chain of dependent loads: a lane per (box,
// output quad, input residue mod 4), the transposed operator read as one
// 16-byte load per input coefficient, and the 4 lanes' partial sums added by
// shuffles.  Measured on 4M Plummer points: 8-19 us per level below ~12,000
// boxes against 23-26 us for the tiles.
__global__ void k_l2l_lanes(int p, int32_t b0, int32_t nbl, const int32_t *__restrict__ parent,
                           const BoxGeo *__restrict__ geo, const float4 *__restrict__ opT,
                           float *L) {
  // 4 consecutive lanes per (box, quad) split the input range (k = k0 + c,
  // k0 + c + 4, ...) and a 2-step shuffle reduction sums them
  const int nc = ncoef(p), ld = coef_pitch(p), nq = ld / 4;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = t >> 2;
  const int c = (int)(t & 3);
  const bool in = g < (int64_t)nbl * nq;
  int32_t b = 0;
  int q = 0;
  if (in) {
    b = b0 + (int32_t)(g / nq);
    q = (int)(g % nq);
  }
  const bool act = in && 4 * q < nc;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (act) {
    const int32_t P = parent[b];
    const int n0 = degree_of(4 * q);
    const float4 *col = opT + (size_t)octant(geo[b]) * nc * nq + q;
    const float *lp = L + (int64_t)P * ld;
    // inputs k = n0^2 + c (mod 4), from the highest degree down (smaller terms first)
    const int kb = n0 * n0 + c;
    for (int k = kb < nc ? kb + (nc - 1 - kb) / 4 * 4 : -1; k >= kb; k -= 4) {
      const float lk = lp[k];
      const float4 w = col[(size_t)k * nq];
      acc.x = fmaf(w.x, lk, acc.x);
      acc.y = fmaf(w.y, lk, acc.y);
      acc.z = fmaf(w.z, lk, acc.z);
      acc.w = fmaf(w.w, lk, acc.w);
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
  }
  if (!act || c != 0) return;
  float4 *out = reinterpret_cast<float4 *>(L + (int64_t)b * ld) + q;
  float4 v = *out;
  v.x += acc.x;
  v.y += acc.y;
  v.z += acc.z;
  v.w += acc.w;
  *out = v;
}

// M2M: each parent of [b0, b0 + nbl) with children sums their parts in child order
__global__ void k_m2m_sum(int p, int32_t b0, int32_t nbl, const int32_t *__restrict__ child,
                          const int32_t *__restrict__ nchild, const float4 *__restrict__ part,
                          float4 *__restrict__ M) {
  const int nq = coef_pitch(p) / 4;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nbl * nq) return;
  const int32_t b = b0 + (int32_t)(i / nq);
  const int q = (int)(i % nq);
  const int32_t nch = nchild[b];
  if (nch == 0) return;
  const int32_t c0 = child[b];
  float4 acc = part[(int64_t)c0 * nq + q];
  for (int c = 1; c < nch; ++c) {
    const float4 v = part[(int64_t)(c0 + c) * nq + q];
    acc.x += v.x;
    acc.y += v.y;
    acc.z += v.z;
    acc.w += v.w;
  }
  M[(int64_t)b * nq + q] = acc;
}

template <typename Tin>
__global__ void k_to_f64(int64_t count, const Tin *__restrict__ in, double *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (double)in[i];
}

// L2P: phi = (1/a) sum L^ R(u), grad = (1/a^2) sum L^ grad_u R(u), u = (x - c)/a.
// With X_n^{-m} = (-1)^m conj(X_n^m) every sum over m is Re(m=0) + 2 Re(m>0);
// the gradient uses d/dz R_n^m = R_{n-1}^m, d/dx R_n^m = (R_{n-1}^{m+1} - R_{n-1}^{m-1})/2,
// d/dy R_n^m = -i (R_{n-1}^{m-1} + R_{n-1}^{m+1})/2, regrouped per R_n^m.
template <typename T, int PT>
__global__ void k_l2p(int p_rt, const int32_t *__restrict__ leaves, const int32_t *__restrict__ first,
                      const int32_t *__restrict__ count, const BoxGeo *__restrict__ geo,
                      const typename V4<T>::type *__restrict__ src,
                      const double *__restrict__ side, const T *__restrict__ L, int64_t n,
                      double *__restrict__ far, int lfar) {
  const int p = PT > 0 ? PT : p_rt;  // compile-time order unrolls the harmonic streams
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ls = reinterpret_cast<T *>(smem_raw);
  const int nc = ncoef(p);
  const int32_t b = leaves[blockIdx.x];
  const BoxGeo g = geo[b];
  const int32_t f = first[b], c = count[b];
  if (g.level < lfar) {  // no far field reaches the levels above lfar
    for (int32_t i = f + threadIdx.x; i < f + c; i += blockDim.x)
      reinterpret_cast<Dbl4 *>(far)[i] = make_dbl4(0.0, 0.0, 0.0, 0.0);
    return;
  }
  for (int k = threadIdx.x; k < nc; k += blockDim.x) Ls[k] = L[(int64_t)b * coef_pitch(p) + k];
  __syncthreads();
  const double a = side[b];
  const T inva = (T)(1.0 / a);
  for (int32_t i = f + threadIdx.x; i < f + c; i += blockDim.x) {
    const typename V4<T>::type s = src[i];
    T phi = 0, gx = 0, gy = 0, gz = 0;
    regular_stream<T>(p, s.x * inva, s.y * inva, s.z * inva, [&](int nn, int m, T re, T im) {
      const T w = m ? T(2) : T(1);
      T ar, ai;
      cget(Ls, p, nn, m, ar, ai);
      phi += w * (ar * re - ai * im);
      if (nn < p) {
        T br, bi, cr, ci;
        cget(Ls, p, nn + 1, m, ar, ai);
        gz += w * (ar * re - ai * im);
        cget(Ls, p, nn + 1, m - 1, br, bi);
        cget(Ls, p, nn + 1, m + 1, cr, ci);
        const T gr = T(0.5) * (br - cr), gi = T(0.5) * (bi - ci);
        gx += w * (gr * re - gi * im);
        const T hr = T(0.5) * (bi + ci), hi = T(-0.5) * (br + cr);
        gy += w * (hr * re - hi * im);
      }
    });
    const double ia = 1.0 / a;
    reinterpret_cast<Dbl4 *>(far)[i] =
        make_dbl4((double)phi * ia, (double)gx * ia * ia, (double)gy * ia * ia,
                     (double)gz * ia * ia);
  }
}

// FP32 L2P, two targets per lane on the paired FP32 instructions.  As for
// M2P below, the gradient is regrouped per regular harmonic: with
// d/dz R_n^m = R_{n-1}^m, d/dx R_n^m = (R_{n-1}^{m+1} - R_{n-1}^{m-1})/2,
// d/dy R_n^m = -i (R_{n-1}^{m-1} + R_{n-1}^{m+1})/2, the coefficient of R_n^m is
//   Gz = L_{n+1}^m,  Gx = (L_{n+1}^{m-1} - L_{n+1}^{m+1})/2,
//   Gy = -i (L_{n+1}^{m-1} + L_{n+1}^{m+1})/2,
// so each warp folds its leaf's local into one 4-vector (L, Gx, Gy, Gz) per
// real slot (the factor 2 of m > 0 and the sign of the imaginary slots
// included), and the evaluation is four dot products sharing one stream.
// One warp per leaf, no block-wide barriers.
constexpr int kL2PWarps = 4;

template <int PT>
__global__ void __launch_bounds__(32 * kL2PWarps, 4)
    k_l2p_f32x2(int p_rt, int64_t nleaves, const int32_t *__restrict__ leaves,
                const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                const BoxGeo *__restrict__ geo, const float4 *__restrict__ src,
                const double *__restrict__ side, const float *__restrict__ L,
                float4 *__restrict__ far, int lfar) {
  const int p = PT > 0 ? PT : p_rt;
  extern __shared__ __align__(16) unsigned char l2p_smem[];
  const int ld = coef_pitch(p), nc = ncoef(p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t li = (int64_t)blockIdx.x * kL2PWarps + warp;
  if (li >= nleaves) return;
  float4 *K = reinterpret_cast<float4 *>(l2p_smem) + (size_t)warp * ld;
  const int32_t b = leaves[li];
  const BoxGeo g = geo[b];
  const int32_t f = first[b], c = count[b];
  float4 *out = far;
  if (g.level < lfar) {  // no far field reaches the levels above lfar
    for (int32_t i = f + lane; i < f + c; i += 32) out[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float *Lb = L + (int64_t)b * ld;
  for (int r = lane; r < nc; r += 32) {
    int n = (int)sqrtf((float)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    const int mm = r - n * n - n, m = mm < 0 ? -mm : mm;
    const bool im_part = mm < 0;
    float ar, ai, br, bi, cr, ci;
    cget(Lb, p, n, m, ar, ai);
    const float k0 = im_part ? ai : ar;
    cget(Lb, p, n + 1, m, ar, ai);
    cget(Lb, p, n + 1, m - 1, br, bi);
    cget(Lb, p, n + 1, m + 1, cr, ci);
    const float kz = im_part ? ai : ar;
    const float kx = 0.5f * (im_part ? (bi - ci) : (br - cr));
    const float ky = im_part ? -0.5f * (br + cr) : 0.5f * (bi + ci);
    const float w = m > 0 ? (im_part ? -2.f : 2.f) : 1.f;
    K[r] = make_float4(w * k0, w * kx, w * ky, w * kz);
  }
  __syncwarp();
  // 1/a and 1/a^2 are powers of two: the scalings below are exact in FP32
  const float inva = (float)(1.0 / side[b]), inva2 = inva * inva;
  for (int32_t tc = 0; tc < c; tc += 64) {
    const int32_t i0 = f + tc + lane, i1 = i0 + 32;
    const bool v0 = tc + lane < c, v1 = tc + lane + 32 < c;
    const float4 s0 = v0 ? src[i0] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 s1 = v1 ? src[i1] : s0;
    float2 fp = make_float2(0.f, 0.f), fx = fp, fy = fp, fz = fp;
    regular_stream2(p, make_float2(s0.x * inva, s1.x * inva), make_float2(s0.y * inva, s1.y * inva),
                    make_float2(s0.z * inva, s1.z * inva), [&](int nn, int m, float2 re, float2 im) {
                      const float4 kp = K[cidx(nn, m)];
                      fp.x = fmaf(kp.x, re.x, fp.x);
                      fp.y = fmaf(kp.x, re.y, fp.y);
                      fx.x = fmaf(kp.y, re.x, fx.x);
                      fx.y = fmaf(kp.y, re.y, fx.y);
                      fy.x = fmaf(kp.z, re.x, fy.x);
                      fy.y = fmaf(kp.z, re.y, fy.y);
                      fz.x = fmaf(kp.w, re.x, fz.x);
                      fz.y = fmaf(kp.w, re.y, fz.y);
                      if (m > 0) {
                        const float4 kn = K[cidx(nn, -m)];
                        fp.x = fmaf(kn.x, im.x, fp.x);
                        fp.y = fmaf(kn.x, im.y, fp.y);
                        fx.x = fmaf(kn.y, im.x, fx.x);
                        fx.y = fmaf(kn.y, im.y, fx.y);
                        fy.x = fmaf(kn.z, im.x, fy.x);
                        fy.y = fmaf(kn.z, im.y, fy.y);
                        fz.x = fmaf(kn.w, im.x, fz.x);
                        fz.y = fmaf(kn.w, im.y, fz.y);
                      }
                    });
    if (v0) out[i0] = make_float4(fp.x * inva, fx.x * inva2, fy.x * inva2, fz.x * inva2);
    if (v1) out[i1] = make_float4(fp.y * inva, fx.y * inva2, fy.y * inva2, fz.y * inva2);
  }
}

// M2P over W lists: phi += (1/a_A) sum M^ I(u), u = (x - c_A)/a_A.  The
// gradient uses d/dz I_n^m = -I_{n+1}^m, d/dx I_n^m = (I_{n+1}^{m+1} - I_{n+1}^{m-1})/2,
// d/dy I_n^m = -i (I_{n+1}^{m+1} + I_{n+1}^{m-1})/2; regrouped per I_n^m they are
// expansions of degree p+1 with coefficients
//   Kz_n^m = -M_{n-1}^m,  Kx_n^m = (M_{n-1}^{m-1} - M_{n-1}^{m+1})/2,
//   Ky_n^m = -i (M_{n-1}^{m-1} + M_{n-1}^{m+1})/2,
// which obey the same X_n^{-m} = (-1)^m conj(X_n^m) symmetry.  A prepass writes
// (M, Kx, Ky, Kz) of every W source box in the real layout, interleaved as
// one 4-vector per coefficient (pitch coef_pitch(p+1)); the evaluation is
// then four dot products that share one harmonic stream.
template <typename T>
__global__ void k_m2p_prep(int p, int64_t nx, const int32_t *__restrict__ xboxes,
                           const T *__restrict__ M, typename V4<T>::type *__restrict__ K) {
  const int ld = coef_pitch(p), ld1 = coef_pitch(p + 1), nc1 = ncoef(p + 1);
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nx * nc1) return;
  const int64_t j = t / nc1;
  const int r = (int)(t % nc1);
  const T *Ma = M + (int64_t)xboxes[j] * ld;
  int n = (int)sqrtf((float)r);
  while (n * n > r) --n;
  while ((n + 1) * (n + 1) <= r) ++n;
  const int mm = r - n * n - n;       // signed index of this slot
  const int m = mm < 0 ? -mm : mm;    // the slot holds Re (mm >= 0) or Im (mm < 0) of X_n^m
  const bool im_part = mm < 0;
  T k0 = 0, kx = 0, ky = 0, kz = 0;
  T ar, ai, br, bi, cr, ci;
  if (n <= p) {
    cget(Ma, p, n, m, ar, ai);
    k0 = im_part ? ai : ar;
  }
  cget(Ma, p, n - 1, m, ar, ai);
  cget(Ma, p, n - 1, m - 1, br, bi);
  cget(Ma, p, n - 1, m + 1, cr, ci);
  kz = -(im_part ? ai : ar);
  kx = T(0.5) * (im_part ? (bi - ci) : (br - cr));
  ky = im_part ? T(-0.5) * (br + cr) : T(0.5) * (bi + ci);
  // a real expansion sums Re(X_n^0 I_n^0) + 2 sum_{m>0} Re(X_n^m I_n^m) and
  // Re(X I) = Re X Re I - Im X Im I: the factor 2 of the m > 0 terms and the
  // sign of the imaginary slots are applied here, once per coefficient, so
  // every term of the evaluation is a plain multiply-add
  const T w = m > 0 ? (im_part ? T(-2) : T(2)) : T(1);
  typename V4<T>::type v;
  v.x = w * k0;
  v.y = w * kx;
  v.z = w * ky;
  v.w = w * kz;
  K[j * ld1 + r] = v;
}

// hi + lo += v without FP64 arithmetic (scarce on this GPU): Knuth's two_sum
// gives the rounding error of hi + v exactly, which is carried in lo
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(v, bv));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// One CTA of 128 threads per target leaf (chunks of 128 targets).  Targets
// sit on lanes; the 4 warps form k = 4 / ceil(targets / 32) replicas that
// split the W list, so all lanes of a warp work on the same source box and
// read its (M, Kx, Ky, Kz) coefficients from shared memory as broadcasts.
// W boxes are staged kM2PStage at a time with their centre offsets and
// scale; per-box sums are taken in T and accumulated in FP64.
constexpr int kM2PThreads = 128;
constexpr int kM2PStage = 16;

template <typename T, int PT>
__global__ void __launch_bounds__(kM2PThreads)
    k_m2p(int p_rt, int nstage, const int32_t *__restrict__ wleaves, const int32_t *__restrict__ woff,
          const int32_t *__restrict__ widx, const int32_t *__restrict__ xslot,
          const int32_t *__restrict__ first, const int32_t *__restrict__ count,
          const BoxGeo *__restrict__ geo, const typename V4<T>::type *__restrict__ src,
          const double *__restrict__ side, const typename V4<T>::type *__restrict__ K, int64_t n,
          double *__restrict__ far) {
  using V = typename V4<T>::type;
  const int p = PT > 0 ? PT : p_rt;  // compile-time order unrolls the harmonic streams
  extern __shared__ __align__(32) unsigned char m2p_smem[];
  V *ks = reinterpret_cast<V *>(m2p_smem);  // [nstage][ld1]
  __shared__ T s_off[kM2PStage][3], s_inva[kM2PStage];
  __shared__ double s_ia[kM2PStage];
  __shared__ int32_t s_slot[kM2PStage];
  __shared__ double red[4][kM2PThreads];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ld1 = coef_pitch(p + 1), nc1 = ncoef(p + 1);
  const int32_t B = wleaves[blockIdx.x];
  const BoxGeo gb = geo[B];
  const double sb = side[B];
  const int32_t f = first[B], c = count[B], e0 = woff[B], e1 = woff[B + 1];
  for (int32_t tc = 0; tc < c; tc += kM2PThreads) {
    const int tcount = min(kM2PThreads, c - tc);
    const int wpr = (tcount + 31) / 32;  // warps per replica
    const int k = 4 / wpr;               // replicas
    const int rep = warp / wpr, ti = (warp - rep * wpr) * 32 + lane;
    const bool act = rep < k && ti < tcount;
    V s;
    s.x = s.y = s.z = s.w = T(0);
    if (act) s = src[f + tc + ti];
    double phi = 0, gx = 0, gy = 0, gz = 0;
    for (int32_t e = e0; e < e1; e += nstage) {
      const int nb = min(nstage, e1 - e);
      __syncthreads();  // the previous batch has been consumed
      if (tid < nb) {
        const int32_t A = widx[e + tid];
        const BoxGeo ga = geo[A];
        const double aa = side[A];
        s_slot[tid] = xslot[A];
        s_off[tid][0] = (T)center_delta(gb.ix, sb, ga.ix, aa);
        s_off[tid][1] = (T)center_delta(gb.iy, sb, ga.iy, aa);
        s_off[tid][2] = (T)center_delta(gb.iz, sb, ga.iz, aa);
        s_inva[tid] = (T)(1.0 / aa);
        s_ia[tid] = 1.0 / aa;
      }
      __syncthreads();
      for (int q = tid; q < nb * nc1; q += kM2PThreads) {
        const int b = q / nc1, r = q - b * nc1;
        ks[b * ld1 + r] = K[(int64_t)s_slot[b] * ld1 + r];
      }
      __syncthreads();
      if (act) {
        for (int b = rep; b < nb; b += k) {
          const V *kb = ks + b * ld1;
          const T inva = s_inva[b];
          T fp = 0, fx = 0, fy = 0, fz = 0;
          irregular_stream<T>(p + 1, (s.x + s_off[b][0]) * inva, (s.y + s_off[b][1]) * inva,
                              (s.z + s_off[b][2]) * inva, [&](int nn, int m, T re, T im) {
                                const V kp = kb[cidx(nn, m)];
                                fp += kp.x * re;
                                fx += kp.y * re;
                                fy += kp.z * re;
                                fz += kp.w * re;
                                if (m > 0) {
                                  const V kn = kb[cidx(nn, -m)];
                                  fp += kn.x * im;
                                  fx += kn.y * im;
                                  fy += kn.z * im;
                                  fz += kn.w * im;
                                }
                              });
          const double ia = s_ia[b];
          phi += (double)fp * ia;
          gx += (double)fx * ia * ia;
          gy += (double)fy * ia * ia;
          gz += (double)fz * ia * ia;
        }
      }
    }
    red[0][tid] = phi;
    red[1][tid] = gx;
    red[2][tid] = gy;
    red[3][tid] = gz;
    __syncthreads();
    if (tid < tcount) {  // target tid: replica r holds it at thread r * 32 * wpr + tid
      double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
      for (int r = 0; r < k; ++r) {
        const int o = r * 32 * wpr + tid;
        a0 += red[0][o];
        a1 += red[1][o];
        a2 += red[2][o];
        a3 += red[3][o];
      }
      const int64_t i = f + tc + tid;
      Dbl4 *fi = reinterpret_cast<Dbl4 *>(far) + i;
      Dbl4 v = *fi;
      v.x += a0;
      v.y += a1;
      v.z += a2;
      v.w += a3;
      *fi = v;
    }
    __syncthreads();  // red is rewritten by the next chunk
  }
}

// FP32 M2P with two targets per lane: the degree p+1 irregular stream runs
// on paired FP32 instructions for both targets, and each staged coefficient
// 4-vector (one 16-byte broadcast load) serves both targets, which halves
// the shared-memory traffic per evaluation (the scalar kernel is bound by
// it).  Up to 256 targets per chunk.  The 128 threads form replicas that
// split the W list: a replica is the smallest multiple of 8 lanes that holds
// the chunk's target pairs, so a leaf of 94 targets runs two replicas of 48
// lanes rather than one of 64 (whole warps left 18 % of the lane slots idle
// on Plummer W leaves).  Lanes of one warp may belong to two replicas; they
// run the same instructions on different staged boxes.  Each box's sums are
// scaled by its 1/a (a power of two, exact) and added to compensated FP32
// totals; FP64 only for the per-target results.
template <int PT>
__global__ void __launch_bounds__(kM2PThreads)
    k_m2p_f32x2(int p_rt, int nstage, const int32_t *__restrict__ wleaves,
                const int32_t *__restrict__ woff, const int32_t *__restrict__ widx,
                const int32_t *__restrict__ xslot, const int32_t *__restrict__ first,
                const int32_t *__restrict__ count, const BoxGeo *__restrict__ geo,
                const float4 *__restrict__ src, const double *__restrict__ side,
                const float4 *__restrict__ K, int64_t n, float4 *__restrict__ far) {
  const int p = PT > 0 ? PT : p_rt;
  extern __shared__ __align__(32) unsigned char m2p_smem[];
  float4 *ks = reinterpret_cast<float4 *>(m2p_smem);  // [nstage][ld1]
  __shared__ float s_off[kM2PStage][3], s_inva[kM2PStage];
  __shared__ int32_t s_slot[kM2PStage];
  __shared__ float red[4][2][kM2PThreads];
  const int tid = threadIdx.x;
  const int ld1 = coef_pitch(p + 1), nc1 = ncoef(p + 1);
  const int32_t B = wleaves[blockIdx.x];
  const BoxGeo gb = geo[B];
  const double sb = side[B];
  const int32_t f = first[B], c = count[B], e0 = woff[B], e1 = woff[B + 1];
  for (int32_t tc = 0; tc < c; tc += 2 * kM2PThreads) {
    const int tcount = min(2 * kM2PThreads, c - tc);
    const int L = ((tcount + 1) / 2 + 7) & ~7;  // lanes per replica
    const int k = max(1, kM2PThreads / L);      // replicas
    const int rep = tid / L, j = tid - rep * L, ti = 2 * j;
    const bool act = rep < k && ti < tcount;
    float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0;
    if (act) {
      s0 = src[f + tc + ti];
      s1 = ti + 1 < tcount ? src[f + tc + ti + 1] : s0;  // a duplicate is evaluated, not stored
    }
    // compensated FP32 totals per target and component, (sum, error) pairs:
    // [component phi, gx, gy, gz][target of the pair]
    float th[4][2] = {}, tl[4][2] = {};
    for (int32_t e = e0; e < e1; e += nstage) {
      const int nb = min(nstage, e1 - e);
      __syncthreads();  // the previous batch has been consumed
      if (tid < nb) {
        const int32_t A = widx[e + tid];
        const BoxGeo ga = geo[A];
        const double aa = side[A];
        s_slot[tid] = xslot[A];
        s_off[tid][0] = (float)center_delta(gb.ix, sb, ga.ix, aa);
        s_off[tid][1] = (float)center_delta(gb.iy, sb, ga.iy, aa);
        s_off[tid][2] = (float)center_delta(gb.iz, sb, ga.iz, aa);
        s_inva[tid] = (float)(1.0 / aa);  // a power of two: exact
      }
      __syncthreads();
      for (int q = tid; q < nb * nc1; q += kM2PThreads) {
        const int b = q / nc1, r = q - b * nc1;
        ks[b * ld1 + r] = K[(int64_t)s_slot[b] * ld1 + r];
      }
      __syncthreads();
      if (act) {
        for (int b = rep; b < nb; b += k) {
          const float4 *kb = ks + b * ld1;
          const float inva = s_inva[b];
          const float ox = s_off[b][0], oy = s_off[b][1], oz = s_off[b][2];
          float2 fp = make_float2(0.f, 0.f), fx = fp, fy = fp, fz = fp;
          irregular_stream2(p + 1, make_float2((s0.x + ox) * inva, (s1.x + ox) * inva),
                            make_float2((s0.y + oy) * inva, (s1.y + oy) * inva),
                            make_float2((s0.z + oz) * inva, (s1.z + oz) * inva),
                            [&](int nn, int m, float2 re, float2 im) {
                              const float4 kp = kb[cidx(nn, m)];
                              fp.x = fmaf(kp.x, re.x, fp.x);
                              fp.y = fmaf(kp.x, re.y, fp.y);
                              fx.x = fmaf(kp.y, re.x, fx.x);
                              fx.y = fmaf(kp.y, re.y, fx.y);
                              fy.x = fmaf(kp.z, re.x, fy.x);
                              fy.y = fmaf(kp.z, re.y, fy.y);
                              fz.x = fmaf(kp.w, re.x, fz.x);
                              fz.y = fmaf(kp.w, re.y, fz.y);
                              if (m > 0) {
                                const float4 kn = kb[cidx(nn, -m)];
                                fp.x = fmaf(kn.x, im.x, fp.x);
                                fp.y = fmaf(kn.x, im.y, fp.y);
                                fx.x = fmaf(kn.y, im.x, fx.x);
                                fx.y = fmaf(kn.y, im.y, fx.y);
                                fy.x = fmaf(kn.z, im.x, fy.x);
                                fy.y = fmaf(kn.z, im.y, fy.y);
                                fz.x = fmaf(kn.w, im.x, fz.x);
                                fz.y = fmaf(kn.w, im.y, fz.y);
                              }
                            });
          const float ia2 = inva * inva;  // exact, as inva
          const float v[4][2] = {{fp.x * inva, fp.y * inva}, {fx.x * ia2, fx.y * ia2},
                                 {fy.x * ia2, fy.y * ia2}, {fz.x * ia2, fz.y * ia2}};
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) two_sum_acc(th[q][h], tl[q][h], v[q][h]);
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[q][h][tid] = th[q][h] + tl[q][h];
    __syncthreads();
    // target pair jj (targets 2 jj, 2 jj + 1): replica r holds it at thread r * L + jj
    if (tid < (tcount + 1) / 2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int u = 2 * tid + h;
        if (u < tcount) {
          float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
          for (int r = 0; r < k; ++r) {
            const int o = r * L + tid;
            a0 += red[0][h][o];
            a1 += red[1][h][o];
            a2 += red[2][h][o];
            a3 += red[3][h][o];
          }
          const int64_t i = f + tc + u;
          float4 *fi = far + i;
          float4 v = *fi;
          v.x += a0;
          v.y += a1;
          v.z += a2;
          v.w += a3;
          *fi = v;
        }
      }
    }
    __syncthreads();  // red is rewritten by the next chunk
  }
}

// final per-target reduction in FP64: far + near per target, gathered into
// the caller's order.  Thread o reads the two 32-byte records of its sorted
// position and writes phi[o], grad[o][:], consecutive threads on consecutive
// addresses.
__global__ void k_combine(int64_t n, const int32_t *__restrict__ iperm,
                          const Dbl4 *__restrict__ far, const Dbl4 *__restrict__ near,
                          double *__restrict__ phi, double *__restrict__ grad) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int64_t i = iperm[o];
  const Dbl4 f = far[i], g = near[i];
  phi[o] = f.x + g.x;
  if (grad) {
    grad[3 * o] = f.y + g.y;
    grad[3 * o + 1] = f.z + g.z;
    grad[3 * o + 2] = f.w + g.w;
  }
}

__global__ void k_adjoint_dx(int64_t n, const double *__restrict__ w, const double *__restrict__ q,
                             const double *__restrict__ gq, const double *__restrict__ gw,
                             double *__restrict__ dx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  const int64_t k = i / 3;
  dx[i] = w[k] * gq[i] + q[k] * gw[i];
}

int warps_for(size_t per_warp) {
  int w = (int)std::min<size_t>(4, (96 * 1024) / std::max<size_t>(per_warp, 1));
  return w < 1 ? 1 : w;
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    FMM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

// ------------------------------------------------------------ launchers
// Calls f(std::integral_constant<int, P>) with P = p for the orders compiled
// with a fixed trip count, else with P = 0 (runtime order).
template <typename F>
void with_order(int p, F &&f) {
  switch (p) {
    case 4: return f(std::integral_constant<int, 4>());
    case 6: return f(std::integral_constant<int, 6>());
    case 8: return f(std::integral_constant<int, 8>());
    case 10: return f(std::integral_constant<int, 10>());
    default: return f(std::integral_constant<int, 0>());
  }
}

template <typename T>
void launch_permute_charges(int64_t n, const int32_t *perm, const double *q,
                            const typename V4<T>::type *pl, typename V4<T>::type *src, cudaStream_t s) {
  if (n == 0) return;
  k_permute_charges<T><<<ceil_div(n, 256), 256, 0, s>>>(n, perm, q, pl, src);
  FMM_LAUNCH_CHECK();
}

template <typename T>
void launch_p2m(int p, int64_t nleaves, const int32_t *leaves, const int32_t *first,
                const int32_t *count, const BoxGeo *geo, const typename V4<T>::type *src, const double *side,
                T *M, double *M64, int coarse, cudaStream_t s) {
  if (nleaves == 0) return;
  size_t per = (size_t)ncoef(p) * 33 * sizeof(T);
  int w = warps_for(per);
  with_order(p, [&](auto PC) {
    constexpr int P = decltype(PC)::value;
    auto kern = k_p2m<T, P>;
    const int wk = reg_accumulate<T, P>() ? 4 : w;
    const size_t sm = per * wk;  // per warp: the (NC x 33) sum buffer
    allow_smem(kern, sm);
    kern<<<ceil_div(nleaves, wk), 32 * wk, sm, s>>>(p, nleaves, leaves, first, count, geo, src, side,
                                                    M, M64, coarse);
  });
  FMM_LAUNCH_CHECK();
}

template <typename T>
void launch_p2l(int p, int64_t nx, const int32_t *xboxes, const int32_t *xoff, const int32_t *xidx,
                const int32_t *first, const int32_t *count, const BoxGeo *geo,
                const typename V4<T>::type *src, const double *side, T *L, cudaStream_t s) {
  if (nx == 0) return;
  size_t per = (size_t)ncoef(p) * 33 * sizeof(T);
  int w = warps_for(per);
  with_order(p, [&](auto PC) {
    constexpr int P = decltype(PC)::value;
    auto kern = k_p2l<T, P>;
    const int wk = reg_accumulate<T, P>() ? 4 : w;
    const size_t sm = per * wk;  // per warp: the (NC x 33) sum buffer
    allow_smem(kern, sm);
    kern<<<ceil_div(nx, wk), 32 * wk, sm, s>>>(p, nx, xboxes, xoff, xidx, first, count, geo, src,
                                               side, L);
  });
  FMM_LAUNCH_CHECK();
}

template <typename Tin, typename Tout, typename Top, typename Tacc>
void launch_m2m(int p, int32_t b0, int32_t nbl, const int32_t *child, const int32_t *nchild,
                const BoxGeo *geo, const Tin *Mc, const Top *ops, Tout *Mp, float *Mp32,
                cudaStream_t s) {
  if (nbl == 0) return;
  int64_t tot = (int64_t)nbl * coef_pitch(p) * 8;
  k_m2m<Tin, Tout, Top, Tacc><<<ceil_div(tot, 128), 128, 0, s>>>(p, b0, nbl, child, nchild, geo, Mc,
                                                                 ops, Mp, Mp32);
  FMM_LAUNCH_CHECK();
}

template <typename Tself, typename Tpar, typename Tout, typename Top, typename Tacc>
void launch_l2l(int p, int32_t b0, int32_t nbl, const int32_t *parent, const BoxGeo *geo,
                const Tself *Lself, const Tpar *Lpar, const Top *ops, Tout *Lout, float *Lout32,
                cudaStream_t s) {
  if (nbl == 0) return;
  int64_t tot = (int64_t)nbl * ncoef(p);
  k_l2l<Tself, Tpar, Tout, Top, Tacc><<<ceil_div(tot, 128), 128, 0, s>>>(p, b0, nbl, parent, geo,
                                                                         Lself, Lpar, ops, Lout,
                                                                         Lout32);
  FMM_LAUNCH_CHECK();
}

namespace {
template <bool L2L>
void launch_trans_oct(int p, int l, int32_t nrows, const int32_t *oct_off, const int32_t *oct_order,
                      const int32_t *parent, const float *opT, const float *in, float *out,
                      cudaStream_t s) {
  if (nrows <= 0) return;
  const int nc = ncoef(p), ld = coef_pitch(p);
  const size_t sm = sizeof(float) * ((size_t)nc * ld + (size_t)nc * kTrPitch);
  const int threads = (8 * (ld / 4) + 31) / 32 * 32;
  // each octant's last tile may be partial: at most 8 tiles more than nrows / kTrRows
  const int64_t grid = ceil_div((int64_t)nrows, (int64_t)kTrRows) + 8;
  allow_smem(k_trans_oct<L2L>, sm);
  k_trans_oct<L2L><<<(unsigned)grid, threads, sm, s>>>(p, l, oct_off, oct_order, parent,
                                                     reinterpret_cast<const float4 *>(opT), in, out);
  FMM_LAUNCH_CHECK();
}
}  // namespace

void launch_octant_groups(int nlevels, const int32_t *level_off_host, int32_t b0, int32_t nb,
                          const BoxGeo *geo, int32_t *oct_off, int32_t *oct_pos, int32_t *oct_order,
                          cudaStream_t s) {
  if (nlevels > kMaxLevels) throw Error(FMM_ERR_UNSUPPORTED, "too many tree levels");
  LevelOffsets lo{};
  lo.n = nlevels;
  for (int l = 0; l <= nlevels; ++l) lo.off[l] = level_off_host[l];
  FMM_CUDA(cudaMemsetAsync(oct_off, 0, sizeof(int32_t) * 9 * (size_t)nlevels, s));
  if (nb > 0) {
    k_oct_count<<<ceil_div(nb, 256), 256, 0, s>>>(b0, nb, lo, geo, oct_off, oct_pos);
    FMM_LAUNCH_CHECK();
  }
  k_oct_scan<<<1, 32, 0, s>>>(lo, oct_off);
  FMM_LAUNCH_CHECK();
  if (nb > 0) {
    k_oct_scatter<<<ceil_div(nb, 256), 256, 0, s>>>(b0, nb, lo, geo, oct_off, oct_pos, oct_order);
    FMM_LAUNCH_CHECK();
  }
}

void launch_m2m_f32q(int p, int l, int32_t b0, int32_t nbl, int32_t nchildren,
                     const int32_t *oct_off, const int32_t *oct_order, const int32_t *child,
                     const int32_t *nchild, const float *opT, float *part, float *M, cudaStream_t s) {
  if (nbl <= 0 || nchildren <= 0) return;
  launch_trans_oct<false>(p, l + 1, nchildren, oct_off, oct_order, nullptr, opT, M, part, s);
  const int64_t tot = (int64_t)nbl * (coef_pitch(p) / 4);
  k_m2m_sum<<<ceil_div(tot, 256), 256, 0, s>>>(p, b0, nbl, child, nchild,
                                              reinterpret_cast<const float4 *>(part),
                                              reinterpret_cast<float4 *>(M));
  FMM_LAUNCH_CHECK();
}

void launch_l2l_f32q(int p, int l, int32_t b0, int32_t nbl, const int32_t *oct_off,
                     const int32_t *oct_order, const int32_t *parent, const BoxGeo *geo,
                     const float *opT, float *L, cudaStream_t s) {
  if (nbl <= 0) return;
  if (nbl < kL2LLanesMaxBoxes) {
    const int64_t tot = (int64_t)nbl * (coef_pitch(p) / 4) * 4;
    k_l2l_lanes<<<ceil_div(tot, 128), 128, 0, s>>>(p, b0, nbl, parent, geo,
                                                   reinterpret_cast<const float4 *>(opT), L);
    FMM_LAUNCH_CHECK();
    return;
  }
  launch_trans_oct<true>(p, l, nbl, oct_off, oct_order, parent, opT, L, L, s);
}

template <typename Tin>
void launch_to_f64(int64_t count, const Tin *in, double *out, cudaStream_t s) {
  if (count == 0) return;
  k_to_f64<Tin><<<ceil_div(count, 256), 256, 0, s>>>(count, in, out);
  FMM_LAUNCH_CHECK();
}

template <typename T>
void launch_l2p(int p, int64_t nleaves, const int32_t *leaves, const int32_t *first,
                const int32_t *count, const BoxGeo *geo, const typename V4<T>::type *src, const double *side,
                const T *L, int64_t n, typename V4<T>::type *far, int lfar, cudaStream_t s) {
  if (nleaves == 0) return;
  if constexpr (sizeof(T) == 4) {
    const size_t sm = (size_t)kL2PWarps * coef_pitch(p) * sizeof(float4);
    with_order(p, [&](auto PC) {
      auto kern = k_l2p_f32x2<decltype(PC)::value>;
      allow_smem(kern, sm);
      kern<<<ceil_div(nleaves, kL2PWarps), 32 * kL2PWarps, sm, s>>>(
          p, nleaves, leaves, first, count, geo, reinterpret_cast<const float4 *>(src), side, L,
          far, lfar);
    });
  } else {
    size_t sm = (size_t)ncoef(p) * sizeof(T);
    with_order(p, [&](auto PC) {
      k_l2p<T, decltype(PC)::value><<<(unsigned)nleaves, 64, sm, s>>>(
          p, leaves, first, count, geo, src, side, L, n, reinterpret_cast<double *>(far), lfar);
    });
  }
  FMM_LAUNCH_CHECK();
}

template <typename T>
void launch_m2p(int p, int64_t nw, const int32_t *wleaves, const int32_t *woff, const int32_t *widx,
                int64_t nx, const int32_t *xboxes, const int32_t *xslot, const int32_t *first,
                const int32_t *count, const BoxGeo *geo, const typename V4<T>::type *src, const double *side,
                const T *M, T *K, int64_t n, typename V4<T>::type *far, cudaStream_t s) {
  if (nw == 0) return;
  using V = typename V4<T>::type;
  V *K4 = reinterpret_cast<V *>(K);  // nx x coef_pitch(p+1) 4-vectors
  const int64_t tot = nx * ncoef(p + 1);
  k_m2p_prep<T><<<ceil_div(tot, 256), 256, 0, s>>>(p, nx, xboxes, M, K4);
  FMM_LAUNCH_CHECK();
  if constexpr (sizeof(T) == 4) {
    // stage as many W boxes as fit in 32 KB (at most kM2PStage)
    const size_t per_box = (size_t)coef_pitch(p + 1) * sizeof(float4);
    const int nstage = (int)std::max<size_t>(1, std::min<size_t>(kM2PStage, (32 << 10) / per_box));
    const size_t sm = nstage * per_box;
    with_order(p, [&](auto PC) {
      auto kern = k_m2p_f32x2<decltype(PC)::value>;
      FMM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      kern<<<(unsigned)nw, kM2PThreads, sm, s>>>(p, nstage, wleaves, woff, widx, xslot, first, count,
                                                 geo, src, side, K4, n, far);
    });
  } else {
    // stage as many W boxes as fit in 64 KB (at most kM2PStage)
    const size_t per_box = (size_t)coef_pitch(p + 1) * sizeof(V);
    const int nstage = (int)std::max<size_t>(1, std::min<size_t>(kM2PStage, (64 << 10) / per_box));
    const size_t sm = nstage * per_box;
    with_order(p, [&](auto PC) {
      auto kern = k_m2p<T, decltype(PC)::value>;
      FMM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      kern<<<(unsigned)nw, kM2PThreads, sm, s>>>(p, nstage, wleaves, woff, widx, xslot, first, count,
                                                 geo, src, side, K4, n, reinterpret_cast<double *>(far));
    });
  }
  FMM_LAUNCH_CHECK();
}

void launch_combine(int64_t n, const int32_t *iperm, const double *far, const double *near,
                    double *phi, double *grad, cudaStream_t s) {
  if (n == 0) return;
  k_combine<<<ceil_div(n, 256), 256, 0, s>>>(n, iperm, reinterpret_cast<const Dbl4 *>(far),
                                             reinterpret_cast<const Dbl4 *>(near), phi, grad);
  FMM_LAUNCH_CHECK();
}

void launch_adjoint_dx(int64_t n, const double *w, const double *q, const double *gq,
                       const double *gw, double *dx, cudaStream_t s) {
  if (n == 0) return;
  k_adjoint_dx<<<ceil_div(3 * n, 256), 256, 0, s>>>(n, w, q, gq, gw, dx);
  FMM_LAUNCH_CHECK();
}

// explicit instantiations
#define FMM_INST_T(T)                                                                              \
  template void launch_permute_charges<T>(int64_t, const int32_t *, const double *,                \
                                          const V4<T>::type *, V4<T>::type *, cudaStream_t);       \
  template void launch_p2m<T>(int, int64_t, const int32_t *, const int32_t *, const int32_t *,     \
                              const BoxGeo *, const V4<T>::type *, const double *, T *, double *, int,     \
                              cudaStream_t);                                                       \
  template void launch_p2l<T>(int, int64_t, const int32_t *, const int32_t *, const int32_t *,     \
                              const int32_t *, const int32_t *, const BoxGeo *,                    \
                              const V4<T>::type *, const double *, T *, cudaStream_t);                     \
  template void launch_l2p<T>(int, int64_t, const int32_t *, const int32_t *, const int32_t *,     \
                              const BoxGeo *, const V4<T>::type *, const double *, const T *, int64_t,     \
                              V4<T>::type *, int, cudaStream_t);                                   \
  template void launch_m2p<T>(int, int64_t, const int32_t *, const int32_t *, const int32_t *,     \
                              int64_t, const int32_t *, const int32_t *, const int32_t *,          \
                              const int32_t *, const BoxGeo *, const V4<T>::type *, const double *, \
                              const T *, T *, int64_t, V4<T>::type *, cudaStream_t);               \
  template void launch_to_f64<T>(int64_t, const T *, double *, cudaStream_t);
FMM_INST_T(float)
FMM_INST_T(double)
#undef FMM_INST_T

template void launch_m2m<double, double, double, double>(int, int32_t, int32_t, const int32_t *,
                                                         const int32_t *, const BoxGeo *,
                                                         const double *, const double *, double *,
                                                         float *, cudaStream_t);
template void launch_m2m<float, float, float, float>(int, int32_t, int32_t, const int32_t *,
                                                     const int32_t *, const BoxGeo *, const float *,
                                                     const float *, float *, float *, cudaStream_t);
template void launch_m2m<float, double, double, double>(int, int32_t, int32_t, const int32_t *,
                                                        const int32_t *, const BoxGeo *,
                                                        const float *, const double *, double *,
                                                        float *, cudaStream_t);
template void launch_l2l<double, double, double, double, double>(int, int32_t, int32_t,
                                                                  const int32_t *, const BoxGeo *,
                                                                  const double *, const double *,
                                                                  const double *, double *, float *,
                                                                  cudaStream_t);
template void launch_l2l<float, float, float, float, float>(int, int32_t, int32_t, const int32_t *,
                                                            const BoxGeo *, const float *,
                                                            const float *, const float *, float *,
                                                            float *, cudaStream_t);
template void launch_l2l<float, double, double, double, double>(int, int32_t, int32_t,
                                                                const int32_t *, const BoxGeo *,
                                                                const float *, const double *,
                                                                const double *, double *, float *,
                                                                cudaStream_t);

}  // namespace fmm

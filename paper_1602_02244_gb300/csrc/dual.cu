// dual.cu -- dual-tree traversal with a multipole acceptance criterion
// (§2.1: Dehnen's dual tree walk, the alternative to fixed interaction
// lists), and the M2L between cells of any two sizes that it produces.
//
// Cells are the octree boxes with their geometric centres as expansion
// centres.  Cell radius r_B = max |x_j - c_B| over B's points.  A pair
// (T, S) of distinct cells is accepted for one M2L from S into T iff
//   r_T + r_S < theta |c_T - c_S|.
// Every quantity in that decision is one IEEE-rounded add, multiply or square
// root in a fixed order (c_T - c_S comes exactly from the integer anchors),
// so the lists are a deterministic function of the points.  A rejected pair
// splits by a rule symmetric in T and S -- both leaves: P2P; one leaf: split
// the other; different levels: split the coarser; same level: split both --
// so (T, S) ends in M2L (P2P) exactly when (S, T) does and the truncated
// operator stays symmetric (the adjoint reuses the forward pass).
//
// The walk runs breadth first from (root, root): one launch per round turns
// the frontier of pending pairs into M2L pairs, P2P leaf pairs and the next
// frontier (warp-aggregated atomic appends).  The pairs are then bucketed by
// target into CSR rows and each row is sorted, which gives the same lists as
// a depth-first walk.  M2L rows go to v_off/v_idx (sources of any level, for
// every box) and P2P rows to u_off/u_idx; W and X are empty.
#include "eval_kernels.cuh"
#include "m2l_config.cuh"
#include "sort.cuh"

namespace fmm {

namespace {

constexpr int kT = 256;

inline int grid(int64_t n) { return n > 0 ? ceil_div(n, kT) : 1; }

// r_B^2 of every box: a warp per leaf walks the leaf's ancestors and takes
// the max of |x_j - c_A|^2 over the leaf's points; every point of a box lies
// in exactly one of its leaves.  Non-negative doubles order like their bit
// patterns, so the max is an integer atomicMax.  FP64 arithmetic is scarce on
// this GPU, so an FP32 pass over the leaf-local coordinates first bounds the
// max; only points within a margin of it (far wider than the FP32 error of
// |x - c_A|^2, about 1e-6 a_A^2) are evaluated in FP64, in the same operation
// order as every other evaluation of the criterion.
__global__ void k_box_radius2(int64_t nleaves, const int32_t *__restrict__ leaves,
                              const BoxGeo *__restrict__ geo, const int32_t *__restrict__ parent,
                              const int32_t *__restrict__ first, const int32_t *__restrict__ count,
                              const double *__restrict__ xyz, const float4 *__restrict__ pl32,
                              const int32_t *__restrict__ bprob, const double *__restrict__ pgeom,
                              const double *__restrict__ side, unsigned long long *__restrict__ r2bits) {
  const int lane = threadIdx.x & 31;
  const int64_t li = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (li >= nleaves) return;
  const int32_t B = leaves[li];
  const int32_t f = first[B], c = count[B];
  const double *lo = pgeom + 8 * (int64_t)bprob[B];
  const BoxGeo gb = geo[B];
  const double ab = side[B];
  const double lomax = fmax(fabs(lo[0]), fmax(fabs(lo[1]), fabs(lo[2]))) + lo[3];
  for (int32_t A = B; A >= 0; A = parent[A]) {
    const BoxGeo g = geo[A];
    const double a = side[A];
    // leaf centre - ancestor centre from the anchors (exact), then FP32
    const float ox = (float)(((double)gb.ix + 0.5) * ab - ((double)g.ix + 0.5) * a);
    const float oy = (float)(((double)gb.iy + 0.5) * ab - ((double)g.iy + 0.5) * a);
    const float oz = (float)(((double)gb.iz + 0.5) * ab - ((double)g.iz + 0.5) * a);
    float mf = 0.f;
    for (int32_t j = f + lane; j < f + c; j += 32) {
      const float4 v = pl32[j];
      const float dx = v.x + ox, dy = v.y + oy, dz = v.z + oz;
      mf = fmaxf(mf, dx * dx + dy * dy + dz * dz);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
    const double margin = 1e-5 * a * a + 1e-12 * lomax * lomax;
    // a leaf whose bound cannot raise the box's current value skips it: most
    // leaves under a coarse box do, so few of them reach the atomic
    const double cur = __longlong_as_double((long long)__ldcg(&r2bits[A]));
    if ((double)mf + margin < cur) continue;
    const float cut = mf - (float)margin;
    // centre = lo + (anchor + 1/2) a: the product is exact, the sum rounds once
    const double cx = __dadd_rn(lo[0], ((double)g.ix + 0.5) * a);
    const double cy = __dadd_rn(lo[1], ((double)g.iy + 0.5) * a);
    const double cz = __dadd_rn(lo[2], ((double)g.iz + 0.5) * a);
    double m = 0.0;
    for (int32_t j = f + lane; j < f + c; j += 32) {
      const float4 v = pl32[j];
      const float dx = v.x + ox, dy = v.y + oy, dz = v.z + oz;
      if (dx * dx + dy * dy + dz * dz < cut) continue;
      const double ex = __dsub_rn(xyz[3 * (int64_t)j], cx);
      const double ey = __dsub_rn(xyz[3 * (int64_t)j + 1], cy);
      const double ez = __dsub_rn(xyz[3 * (int64_t)j + 2], cz);
      const double s = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
      m = fmax(m, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m > cur) atomicMax(&r2bits[A], (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_radius_sqrt(int64_t nb, const unsigned long long *__restrict__ r2bits,
                              double *__restrict__ r) {
  const int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b < nb) r[b] = __dsqrt_rn(__longlong_as_double((long long)r2bits[b]));
}

__device__ __forceinline__ bool mac_accept(const BoxGeo &gt, double at, const BoxGeo &gs, double as,
                                           double rt, double rs, double theta) {
  // c_T - c_S per axis: both centres are dyadic, the difference is exact
  const double dx = ((double)gt.ix + 0.5) * at - ((double)gs.ix + 0.5) * as;
  const double dy = ((double)gt.iy + 0.5) * at - ((double)gs.iy + 0.5) * as;
  const double dz = ((double)gt.iz + 0.5) * at - ((double)gs.iz + 0.5) * as;
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return __dadd_rn(rt, rs) < __dmul_rn(theta, __dsqrt_rn(d2));
}

// Reserve k slots of a counter for this lane; the warp issues one atomic.
// Every lane of the warp calls it (k = 0 for idle lanes).
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long *ctr, int k, int lane) {
  int incl = k;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total > 0) base = atomicAdd(ctr, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + (unsigned long long)(incl - k);
}

// One round of the walk.  cnt[0] next frontier, cnt[1] M2L pairs, cnt[2] P2P
// pairs (running totals); an append past a buffer's capacity is counted but
// not written, and the host reruns the round with larger buffers.
__global__ void k_dual_round(int64_t nf, const int2 *__restrict__ F, const BoxGeo *__restrict__ geo,
                             const double *__restrict__ side, const double *__restrict__ radius,
                             const int32_t *__restrict__ child, const int32_t *__restrict__ nchild,
                             double theta, int2 *__restrict__ next, int64_t cap_next,
                             int2 *__restrict__ m2l, int64_t cap_m2l, int2 *__restrict__ p2p,
                             int64_t cap_p2p, unsigned long long *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < nf; i0 += stride) {
    const int64_t i = i0 + lane;
    int kind = 0, nt = 0, ns = 0;  // kind 1 M2L, 2 P2P, 3 split
    int32_t T = 0, S = 0;
    bool splitT = false, splitS = false;
    if (i < nf) {
      const int2 pr = F[i];
      T = pr.x;
      S = pr.y;
      const BoxGeo gt = geo[T], gs = geo[S];
      const int ct = nchild[T], cs = nchild[S];
      if (T != S && mac_accept(gt, side[T], gs, side[S], radius[T], radius[S], theta)) {
        kind = 1;
      } else if (ct == 0 && cs == 0) {
        kind = 2;
      } else {
        kind = 3;
        if (ct == 0) splitS = true;
        else if (cs == 0) splitT = true;
        else if (gt.level != gs.level) (gt.level < gs.level ? splitT : splitS) = true;
        else splitT = splitS = true;
        nt = splitT ? ct : 1;
        ns = splitS ? cs : 1;
      }
    }
    const int knext = kind == 3 ? nt * ns : 0;
    const unsigned long long bm = warp_reserve(&cnt[1], kind == 1, lane);
    const unsigned long long bp = warp_reserve(&cnt[2], kind == 2, lane);
    const unsigned long long bn = warp_reserve(&cnt[0], knext, lane);
    if (kind == 1 && bm < (unsigned long long)cap_m2l) m2l[bm] = make_int2(T, S);
    if (kind == 2 && bp < (unsigned long long)cap_p2p) p2p[bp] = make_int2(T, S);
    if (kind == 3 && bn + knext <= (unsigned long long)cap_next) {
      const int32_t t0 = splitT ? child[T] : T, s0 = splitS ? child[S] : S;
      int w = 0;
      for (int a = 0; a < nt; ++a)
        for (int b = 0; b < ns; ++b) next[bn + w++] = make_int2(t0 + a, s0 + b);
    }
  }
}

__global__ void k_row_count(int64_t np, const int2 *__restrict__ pairs, int32_t *__restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i < np) atomicAdd(&cnt[pairs[i].x], 1);
}

__global__ void k_row_fill(int64_t np, const int2 *__restrict__ pairs, const int32_t *__restrict__ off,
                           int32_t *__restrict__ fill, int32_t *__restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= np) return;
  const int2 pr = pairs[i];
  idx[off[pr.x] + atomicAdd(&fill[pr.x], 1)] = pr.y;
}

// Sort every CSR row ascending: a warp per row, a bitonic network over the
// row padded to a power of two in shared memory; the rare rows longer than
// kRowSortMax are sorted in place by one thread.
constexpr int kRowSortWarps = 4, kRowSortMax = 2048;

__global__ void __launch_bounds__(32 * kRowSortWarps)
    k_row_sort(int64_t nb, const int32_t *__restrict__ off, int32_t *__restrict__ idx) {
  __shared__ int32_t buf_all[kRowSortWarps][kRowSortMax];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t *buf = buf_all[warp];
  for (int64_t b = (int64_t)blockIdx.x * kRowSortWarps + warp; b < nb;
       b += (int64_t)gridDim.x * kRowSortWarps) {
    const int32_t o = off[b], n = off[b + 1] - o;
    if (n < 2) continue;
    if (n > kRowSortMax) {
      if (lane == 0) sort_run(idx + o, n);
      continue;
    }
    int P2 = 32;
    while (P2 < n) P2 <<= 1;
    for (int i = lane; i < P2; i += 32) buf[i] = i < n ? idx[o + i] : 0x7fffffff;
    __syncwarp();
    for (int k = 2; k <= P2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < P2; i += 32) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const int32_t x = buf[i], y = buf[ixj];
            if (((i & k) == 0) == (x > y)) {
              buf[i] = y;
              buf[ixj] = x;
            }
          }
        }
        __syncwarp();
      }
    for (int i = lane; i < n; i += 32) idx[o + i] = buf[i];
    __syncwarp();
  }
}

// Split each M2L row into the pairs the fixed-offset operators of the M2L
// tiles cover (same level, 2 <= max|d| <= 3, inside the 6x6x6 slot window of
// the target's octant parity; the tensor-core path) and the rest, keeping
// the ascending order of both.
template <bool kFill>
__global__ void k_dual_split(int64_t nb, const int32_t *__restrict__ off, const int32_t *__restrict__ idx,
                             const BoxGeo *__restrict__ geo, int32_t *__restrict__ tcnt,
                             int32_t *__restrict__ gcnt, const int32_t *__restrict__ toff,
                             int32_t *__restrict__ tidx, const int32_t *__restrict__ goff,
                             int32_t *__restrict__ gidx) {
  const int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b >= nb) return;
  const BoxGeo gt = geo[b];
  const int px = gt.ix & 1, py = gt.iy & 1, pz = gt.iz & 1;
  int32_t kt = 0, kg = 0;
  for (int32_t e = off[b]; e < off[b + 1]; ++e) {
    const int32_t S = idx[e];
    const BoxGeo gs = geo[S];
    const int dx = gs.ix - gt.ix, dy = gs.iy - gt.iy, dz = gs.iz - gt.iz;
    const int cheb = max(abs(dx), max(abs(dy), abs(dz)));
    const bool tc = gs.level == gt.level && gt.level >= 2 && cheb >= 2 && cheb <= 3 &&
                    (unsigned)(dx + 2 + px) < 6u && (unsigned)(dy + 2 + py) < 6u &&
                    (unsigned)(dz + 2 + pz) < 6u;
    if (tc) {
      if (kFill) tidx[toff[b] + kt] = S;
      ++kt;
    } else {
      if (kFill) gidx[goff[b] + kg] = S;
      ++kg;
    }
  }
  if (!kFill) {
    tcnt[b] = kt;
    gcnt[b] = kg;
  }
}

// CSR rows (nb + 1 offsets, sources ascending) from unordered (target,
// source) pairs; returns the number of pairs
int64_t pairs_to_rows(fmm_plan_impl &P, const int2 *pairs, int64_t np, DBuf<int32_t> &off,
                      DBuf<int32_t> &idx) {
  cudaStream_t s = P.stream;
  const int64_t nb = P.nboxes;
  P.s_i32a.resize(nb, s);
  FMM_CUDA(cudaMemsetAsync(P.s_i32a.p, 0, sizeof(int32_t) * nb, s));
  if (np > 0) {
    k_row_count<<<grid(np), kT, 0, s>>>(np, pairs, P.s_i32a.p);
    FMM_LAUNCH_CHECK();
  }
  off.resize(nb + 1, s);
  scan_exclusive(P.s_i32a.p, off.p, nb, off.p + nb, P.s_scan, s);
  idx.resize(np > 0 ? np : 1, s);
  FMM_CUDA(cudaMemsetAsync(P.s_i32a.p, 0, sizeof(int32_t) * nb, s));
  if (np > 0) {
    k_row_fill<<<grid(np), kT, 0, s>>>(np, pairs, off.p, P.s_i32a.p, idx.p);
    FMM_LAUNCH_CHECK();
    k_row_sort<<<(unsigned)std::min<int64_t>(ceil_div(nb, (int64_t)kRowSortWarps), 152 * 16),
                 32 * kRowSortWarps, 0, s>>>(nb, off.p, idx.p);
    FMM_LAUNCH_CHECK();
  }
  return np;
}

// ------------------------------------------------------------------ M2L
// L^_n^m(T) += (a_T/l)^{n+1} (-1)^{n+m} sum_{k,l'} (a_S/l)^k M^_k^l'(S) I_{n+k}^{l'-m}(d/l)
// with d = c_T - c_S and l = max(a_T, a_S) (scale-free coefficients of each
// box's own side; the irregular addition theorem of the solid harmonics).
// Cells never overlap, so |d| > l/2, and the walk bounds |d|/l from above:
// the harmonics stay in range in FP32.  Folding l' < 0 into l' > 0 with
// X_n^{-m} = (-1)^m conj(X_n^m):
//   M_k^{-l'} I_j^{-l'-m} = (-1)^m conj(M_k^l' I_j^{l'+m}),
// and l' + m <= k + n = j keeps every index inside the table.
// 2^e as T without FP64 work (FP64 runs at a small fraction of the FP32 rate
// on this part): built from the exponent bits, zero below the normal range
// (such terms are far below the FP32 rounding of the result).
template <typename T>
__device__ __forceinline__ T pow2(int e);
template <>
__device__ __forceinline__ float pow2<float>(int e) {
  return e < -126 ? 0.f : __int_as_float((127 + e) << 23);
}
template <>
__device__ __forceinline__ double pow2<double>(int e) {
  return e < -1022 ? 0.0 : __longlong_as_double((long long)(1023 + e) << 52);
}

// One block per target box; thread t < (p+1)(p+2)/2 owns output (n, m >= 0).
// Per source the first 2p+1 threads build the columns m and -m of I_j^i
// (|i| <= j <= 2p) in shared memory and the block stages the source's scaled
// multipole; each thread then reads the table at fixed offsets from two base
// addresses (no branches in the inner loop).  The table is column-major with
// a row pitch chosen so that the lanes' base addresses fall in different
// shared-memory banks (at most two lanes per bank for p = 4..10, against up
// to seven with the plain pitch).
__host__ __device__ constexpr int dual_pitch(int p) {
  return p == 4 ? 13 : p == 6 ? 13 : p == 8 ? 18 : p == 10 ? 23 : 2 * p + 1;
}

template <typename T, int PT>
__global__ void k_m2l_dual(int p_rt, const int32_t *__restrict__ off, const int32_t *__restrict__ idx,
                           const BoxGeo *__restrict__ geo, const T *__restrict__ M,
                           T *__restrict__ L, int ld, int accumulate) {
  extern __shared__ __align__(16) unsigned char dual_smem[];
  const int p = PT > 0 ? PT : p_rt;
  const int P2 = 2 * p, R = dual_pitch(p);  // I_j^i at (i + 2p) R + j
  const int nI = (2 * P2 + 1) * R;
  const int nc = (p + 1) * (p + 1);
  T *sIr = reinterpret_cast<T *>(dual_smem), *sIi = sIr + nI, *sM = sIi + nI;
  const int tid = threadIdx.x;
  const int32_t B = blockIdx.x;
  const int nout = (p + 1) * (p + 2) / 2;
  const bool act = tid < nout;
  int on = 0;
  while ((on + 1) * (on + 2) / 2 <= tid && on < p) ++on;
  const int om = act ? tid - on * (on + 1) / 2 : 0;
  const T sgm = (om & 1) ? T(-1) : T(1);
  // I_{on+k}^{l-om} at a + l R + k and I_{on+k}^{l+om} at b + l R + k
  const T *ar = sIr + (P2 - om) * R + on, *ai = sIi + (P2 - om) * R + on;
  const T *br = sIr + (P2 + om) * R + on, *bi = sIi + (P2 + om) * R + on;
  T accr = T(0), acci = T(0);
  const BoxGeo gt = geo[B];
  for (int32_t e = off[B]; e < off[B + 1]; ++e) {
    const int32_t S = idx[e];
    const BoxGeo gs = geo[S];
    // sides relative to l = max(a_T, a_S): a_X / l = 2^-(level_X - min level)
    const int lmin = min(gt.level, gs.level);
    const int eT = gt.level - lmin, eS = gs.level - lmin;
    __syncthreads();  // the previous source's tables are no longer read
    if (tid <= P2) {
      // d / l per axis = ((2 i_T + 1) 2^(E - eT) - (2 i_S + 1) 2^(E - eS)) 2^-(E + 1),
      // E = max(eT, eS): an exact integer, rounded once to T, times a power of 2
      const int E = max(eT, eS);
      const T h = pow2<T>(-E - 1);
      const T x = (T)(((2 * (int64_t)gt.ix + 1) << (E - eT)) - ((2 * (int64_t)gs.ix + 1) << (E - eS))) * h;
      const T y = (T)(((2 * (int64_t)gt.iy + 1) << (E - eT)) - ((2 * (int64_t)gs.iy + 1) << (E - eS))) * h;
      const T z = (T)(((2 * (int64_t)gt.iz + 1) << (E - eT)) - ((2 * (int64_t)gs.iz + 1) << (E - eS))) * h;
      const T r2 = x * x + y * y + z * z;
      const T inv = T(1) / r2;
      const int m = tid;
      const T sg = (m & 1) ? T(-1) : T(1);
      T dre = T(1) / sqrt(r2), dim = T(0);
      for (int i = 1; i <= m; ++i) {
        const T c = -T(2 * i - 1) * inv;
        const T nre = c * (x * dre - y * dim), nim = c * (x * dim + y * dre);
        dre = nre;
        dim = nim;
      }
      T pre = T(0), pim = T(0), cre = dre, cim = dim;
      for (int n = m; n <= P2; ++n) {
        if (n > m) {
          const T a = T(2 * n - 1) * z, b = T((n - 1) * (n - 1) - m * m);
          const T nre = (a * cre - b * pre) * inv, nim = (a * cim - b * pim) * inv;
          pre = cre;
          pim = cim;
          cre = nre;
          cim = nim;
        }
        sIr[(P2 + m) * R + n] = cre;
        sIi[(P2 + m) * R + n] = cim;
        sIr[(P2 - m) * R + n] = sg * cre;  // I_n^{-m} = (-1)^m conj(I_n^m)
        sIi[(P2 - m) * R + n] = -sg * cim;
      }
    }
    for (int k = tid; k < nc; k += blockDim.x) {
      int deg = 0;
      while ((deg + 1) * (deg + 1) <= k) ++deg;
      sM[k] = M[(int64_t)S * ld + k] * pow2<T>(-eS * deg);
    }
    __syncthreads();
    if (act) {
      T sr = T(0), si = T(0);
#pragma unroll
      for (int k = 0; k <= (PT > 0 ? PT : kMaxOrder); ++k) {
        if (PT == 0 && k > p) break;
        const T m0 = sM[k * k + k];
        sr += m0 * ar[k];  // l' = 0: M_k^0 I_j^{-m}
        si += m0 * ai[k];
#pragma unroll
        for (int l = 1; l <= k; ++l) {
          const T mr = sM[k * k + k + l], mi = sM[k * k + k - l];
          const int o = l * R + k;
          const T a_r = ar[o], a_i = ai[o], b_r = br[o], b_i = bi[o];
          const T u = a_r + sgm * b_r, v = a_i + sgm * b_i;  // A + (-1)^m B
          const T w = a_i - sgm * b_i, x = a_r - sgm * b_r;  // for the imaginary part
          sr += mr * u - mi * v;
          si += mr * w + mi * x;
        }
      }
      const T sc = (((on + om) & 1) ? T(-1) : T(1)) * pow2<T>(-eT * (on + 1));
      accr += sc * sr;
      acci += sc * si;
    }
  }
  T *out = L + (int64_t)B * ld;
  if (act) {
    if (accumulate) {
      accr += out[cidx(on, om)];
      if (om > 0) acci += out[cidx(on, -om)];
    }
    out[cidx(on, om)] = accr;
    if (om > 0) out[cidx(on, -om)] = acci;
  }
  for (int k = nc + tid; k < ld; k += blockDim.x) out[k] = T(0);
}

}  // namespace

void build_dual_lists(fmm_plan_impl &P) {
  cudaStream_t s = P.stream;
  const int64_t nb = P.nboxes;
  P.nw = P.nx = 0;
  P.nxboxes = P.nwleaves = P.nm2l_tiles = 0;
  // cell radii
  DBuf<uint64_t> &r2 = P.s_u64a;
  r2.resize(nb, s);
  FMM_CUDA(cudaMemsetAsync(r2.p, 0, sizeof(uint64_t) * nb, s));
  constexpr int kWarps = 8;
  k_box_radius2<<<(unsigned)ceil_div(P.nleaves, (int64_t)kWarps), 32 * kWarps, 0, s>>>(
      P.nleaves, P.leaves.p, P.box_geo.p, P.box_parent.p, P.box_first.p, P.box_count.p,
      P.xyz_sorted.p, P.pl32.p, P.box_prob.p, P.prob_geom.p, P.box_side.p,
      reinterpret_cast<unsigned long long *>(r2.p));
  FMM_LAUNCH_CHECK();
  P.radius.resize(nb, s);
  k_radius_sqrt<<<grid(nb), kT, 0, s>>>(nb, reinterpret_cast<unsigned long long *>(r2.p), P.radius.p);
  FMM_LAUNCH_CHECK();

  // breadth-first walk from (root, root) of every problem
  const int64_t nroots = P.level_off.size() > 1 ? P.level_off[1] : 0;
  std::vector<int2> roots((size_t)nroots);
  for (int64_t r = 0; r < nroots; ++r) roots[(size_t)r] = make_int2((int)r, (int)r);
  P.dt_a.resize(std::max<int64_t>(nroots, 1024), s);
  FMM_CUDA(cudaMemcpyAsync(P.dt_a.p, roots.data(), sizeof(int2) * nroots, cudaMemcpyHostToDevice, s));
  P.dt_b.resize(std::max<int64_t>(64 * nroots, 1 << 16), s);
  P.dt_m2l.resize(std::max<int64_t>(64 * nb, 1 << 16), s);
  P.dt_p2p.resize(std::max<int64_t>(16 * P.nleaves, 1 << 16), s);
  P.dt_cnt.resize(3, s);
  unsigned long long h[3] = {0, 0, 0};
  int64_t nf = nroots, nm = 0, np = 0;
  while (nf > 0) {
    h[0] = 0;
    h[1] = (unsigned long long)nm;
    h[2] = (unsigned long long)np;
    FMM_CUDA(cudaMemcpyAsync(P.dt_cnt.p, h, sizeof h, cudaMemcpyHostToDevice, s));
    const int blocks = (int)std::min<int64_t>(ceil_div(nf, (int64_t)kT), 152 * 8);
    k_dual_round<<<blocks, kT, 0, s>>>(nf, P.dt_a.p, P.box_geo.p, P.box_side.p, P.radius.p,
                                       P.box_child.p, P.box_nchild.p, P.theta, P.dt_b.p,
                                       (int64_t)P.dt_b.cap, P.dt_m2l.p, (int64_t)P.dt_m2l.cap,
                                       P.dt_p2p.p, (int64_t)P.dt_p2p.cap, P.dt_cnt.p);
    FMM_LAUNCH_CHECK();
    FMM_CUDA(cudaMemcpyAsync(h, P.dt_cnt.p, sizeof h, cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    const int64_t nn = (int64_t)h[0], nm1 = (int64_t)h[1], np1 = (int64_t)h[2];
    bool redo = false;
    if (nn > (int64_t)P.dt_b.cap) {
      P.dt_b.resize((size_t)nn, s);  // contents are rewritten by the rerun
      redo = true;
    }
    if (nm1 > (int64_t)P.dt_m2l.cap) {
      P.dt_m2l.grow((size_t)nm1, (size_t)nm, s);
      redo = true;
    }
    if (np1 > (int64_t)P.dt_p2p.cap) {
      P.dt_p2p.grow((size_t)np1, (size_t)np, s);
      redo = true;
    }
    if (redo) continue;  // the same round again: every slot it appends is rewritten
    nm = nm1;
    np = np1;
    nf = nn;
    std::swap(P.dt_a, P.dt_b);
  }
  P.nv = pairs_to_rows(P, P.dt_m2l.p, nm, P.v_off, P.v_idx);
  P.nu = pairs_to_rows(P, P.dt_p2p.p, np, P.u_off, P.u_idx);
  for (DBuf<int32_t> *o : {&P.w_off, &P.x_off}) {  // empty W and X rows
    o->resize(nb + 1, s);
    FMM_CUDA(cudaMemsetAsync(o->p, 0, sizeof(int32_t) * (nb + 1), s));
  }
  P.w_idx.resize(1, s);
  P.x_idx.resize(1, s);

  // mixed precision, orders with fixed-offset M2L tiles: the pairs those
  // tiles cover run there (tensor cores), the rest in the per-pair kernel
  P.ndt_t = P.ndt_g = 0;
  if (P.precision == FMM_MIXED && P.order <= kM2LStagedMaxOrder) {
    P.s_i32a.resize(nb, s);
    P.s_i32b.resize(nb, s);
    k_dual_split<false><<<grid(nb), kT, 0, s>>>(nb, P.v_off.p, P.v_idx.p, P.box_geo.p, P.s_i32a.p,
                                                P.s_i32b.p, nullptr, nullptr, nullptr, nullptr);
    FMM_LAUNCH_CHECK();
    P.dt_toff.resize(nb + 1, s);
    P.dt_goff.resize(nb + 1, s);
    scan_exclusive(P.s_i32a.p, P.dt_toff.p, nb, P.dt_toff.p + nb, P.s_scan, s);
    scan_exclusive(P.s_i32b.p, P.dt_goff.p, nb, P.dt_goff.p + nb, P.s_scan, s);
    P.ndt_t = read_scalar(P.dt_toff.p + nb, s);
    P.ndt_g = read_scalar(P.dt_goff.p + nb, s);
    P.dt_tidx.resize(P.ndt_t > 0 ? P.ndt_t : 1, s);
    P.dt_gidx.resize(P.ndt_g > 0 ? P.ndt_g : 1, s);
    k_dual_split<true><<<grid(nb), kT, 0, s>>>(nb, P.v_off.p, P.v_idx.p, P.box_geo.p, nullptr,
                                               nullptr, P.dt_toff.p, P.dt_tidx.p, P.dt_goff.p,
                                               P.dt_gidx.p);
    FMM_LAUNCH_CHECK();
    build_m2l_tiles(P);
  }
  FMM_CUDA(cudaStreamSynchronize(s));  // `roots` is a host temporary
}

template <typename T>
void launch_m2l_dual(int p, int64_t nb, const int32_t *off, const int32_t *idx, const BoxGeo *geo,
                     const T *M, T *L, bool accumulate, cudaStream_t s) {
  if (nb <= 0) return;
  const int nout = (p + 1) * (p + 2) / 2;
  const int threads = std::max(64, (nout + 31) / 32 * 32);
  const size_t nI = (size_t)(4 * p + 1) * dual_pitch(p);
  const size_t smem = sizeof(T) * (2 * nI + (size_t)(p + 1) * (p + 1));
  auto go = [&](auto kern) {
    if (smem > 48 * 1024) FMM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)nb, threads, smem, s>>>(p, off, idx, geo, M, L, coef_pitch(p), accumulate ? 1 : 0);
  };
  switch (p) {
    case 4: go(k_m2l_dual<T, 4>); break;
    case 6: go(k_m2l_dual<T, 6>); break;
    case 8: go(k_m2l_dual<T, 8>); break;
    case 10: go(k_m2l_dual<T, 10>); break;
    default: go(k_m2l_dual<T, 0>); break;
  }
  FMM_LAUNCH_CHECK();
}

template void launch_m2l_dual<double>(int, int64_t, const int32_t *, const int32_t *, const BoxGeo *,
                                      const double *, double *, bool, cudaStream_t);
template void launch_m2l_dual<float>(int, int64_t, const int32_t *, const int32_t *, const BoxGeo *,
                                     const float *, float *, bool, cudaStream_t);

}  // namespace fmm

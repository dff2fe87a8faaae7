// tree.cu -- hierarchy of the FMM on the GPU: root cube, Morton keys (§3.1
// 3D->1D locality mapping), stable radix sort, adaptive octree level by
// level, colleagues, and the U/V/W/X interaction lists (§2.2: the
// interaction list holds the children of the parent's neighbours that are
// not neighbours, at most 189; U/W/X are the adaptive lists of the cited
// kernel-independent FMM).
//
// All of it is integer work and bit-exact: the quantisation uses
// round-to-nearest FP64 subtract then an exact power-of-two scale, boxes are
// numbered by (level, key) and every list is sorted by box number.
#include <algorithm>
#include <memory>
#include <utility>

#include "m2l_config.cuh"

#include "plan.cuh"
#include "sort.cuh"

namespace fmm {

namespace {

constexpr int kT = 256;

// ------------------------------------------------------------ root cube
__global__ void k_bbox_partial(const double *__restrict__ xyz, int64_t n, double *partial) {
  __shared__ double smin[3][kT], smax[3][kT];
  __shared__ int sbad[kT];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    for (int a = 0; a < 3; ++a) {
      double v = xyz[3 * i + a];
      if (!isfinite(v)) bad = 1;
      mn[a] = fmin(mn[a], v);
      mx[a] = fmax(mx[a], v);
    }
  }
  for (int a = 0; a < 3; ++a) {
    smin[a][threadIdx.x] = mn[a];
    smax[a][threadIdx.x] = mx[a];
  }
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + o]);
        smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + o]);
      }
      sbad[threadIdx.x] |= sbad[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) {
      partial[7 * blockIdx.x + a] = smin[a][0];
      partial[7 * blockIdx.x + 3 + a] = smax[a][0];
    }
    partial[7 * blockIdx.x + 6] = sbad[0];
  }
}

__global__ void k_bbox_final(const double *partial, int nb, double *geom) {
  // one CTA of kT threads reduces the per-CTA partials
  __shared__ double smin[3][kT], smax[3][kT], sbad[kT];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  double bad = 0;
  for (int b = threadIdx.x; b < nb; b += kT) {
    for (int a = 0; a < 3; ++a) {
      mn[a] = fmin(mn[a], partial[7 * b + a]);
      mx[a] = fmax(mx[a], partial[7 * b + 3 + a]);
    }
    bad = fmax(bad, partial[7 * b + 6]);
  }
  for (int a = 0; a < 3; ++a) {
    smin[a][threadIdx.x] = mn[a];
    smax[a][threadIdx.x] = mx[a];
  }
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + o]);
        smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + o]);
      }
      sbad[threadIdx.x] = fmax(sbad[threadIdx.x], sbad[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) ext = fmax(ext, smax[a][0] - smin[a][0]);
  double D = 1.0;
  if (ext > 0.0) {
    int e;
    frexp(ext, &e);  // ext = f 2^e with f in [0.5,1): 2^e is the smallest power of two > ext
    D = ldexp(1.0, e);
  }
  for (int a = 0; a < 3; ++a) geom[a] = smin[a][0];
  geom[3] = D;
  geom[4] = sbad[0];
  geom[5] = ldexp(1.0, kMaxDepth) / D;  // quantisation scale, a power of two
}

// one CTA per problem of a batch: root cube of its points (same rule as above)
__global__ void k_bbox_problems(const double *__restrict__ xyz, const int64_t *__restrict__ off,
                                double *__restrict__ geom) {
  __shared__ double smin[3][kT], smax[3][kT];
  __shared__ int sbad[kT];
  const int b = blockIdx.x;
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  for (int64_t i = off[b] + threadIdx.x; i < off[b + 1]; i += kT)
    for (int a = 0; a < 3; ++a) {
      double v = xyz[3 * i + a];
      if (!isfinite(v)) bad = 1;
      mn[a] = fmin(mn[a], v);
      mx[a] = fmax(mx[a], v);
    }
  for (int a = 0; a < 3; ++a) {
    smin[a][threadIdx.x] = mn[a];
    smax[a][threadIdx.x] = mx[a];
  }
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      for (int a = 0; a < 3; ++a) {
        smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + o]);
        smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + o]);
      }
      sbad[threadIdx.x] |= sbad[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double *g = geom + 8 * b;
  if (off[b + 1] == off[b]) {  // empty problem
    g[0] = g[1] = g[2] = 0.0;
    g[3] = 1.0;
    g[4] = 0.0;
    g[5] = ldexp(1.0, kMaxDepth);
    return;
  }
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) ext = fmax(ext, smax[a][0] - smin[a][0]);
  double D = 1.0;
  if (ext > 0.0) {
    int e;
    frexp(ext, &e);
    D = ldexp(1.0, e);
  }
  for (int a = 0; a < 3; ++a) g[a] = smin[a][0];
  g[3] = D;
  g[4] = sbad[0];
  g[5] = ldexp(1.0, kMaxDepth) / D;  // quantisation scale, a power of two
}

__device__ __forceinline__ int problem_of(int64_t i, const int64_t *__restrict__ off, int nprob) {
  int lo = 0, hi = nprob - 1;  // last b with off[b] <= i
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Morton key of every point in its own problem's root cube (geom: 8 doubles
// per problem; one problem when off == nullptr)
__global__ void k_morton(const double *__restrict__ xyz, int64_t n, const double *__restrict__ geom,
                         const int64_t *__restrict__ off, int nprob, uint64_t *__restrict__ keys,
                         int32_t *__restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  const double *g = geom + (off ? 8 * problem_of(i, off, nprob) : 0);
  const double s = g[5];  // 2^21 / D, a power of two: the product below is exact
  const double top = (double)((1u << kMaxDepth) - 1u);
  uint32_t q[3];
  for (int a = 0; a < 3; ++a) {
    double t = floor(__dmul_rn(__dsub_rn(xyz[3 * i + a], g[a]), s));
    t = fmin(fmax(t, 0.0), top);
    q[a] = (uint32_t)t;
  }
  keys[i] = morton3(q[0], q[1], q[2]);
  perm[i] = (int32_t)i;
}

__global__ void k_problem_keys(int64_t n, const int32_t *__restrict__ perm,
                               const int64_t *__restrict__ off, int nprob,
                               uint64_t *__restrict__ pk, int32_t *__restrict__ idx) {
  int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  pk[i] = (uint64_t)problem_of(perm[i], off, nprob);
  idx[i] = (int32_t)i;
}

__global__ void k_apply_perm(int64_t n, const int32_t *__restrict__ sigma,
                             const uint64_t *__restrict__ kin, const int32_t *__restrict__ pin,
                             uint64_t *__restrict__ kout, int32_t *__restrict__ pout) {
  int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  kout[i] = kin[sigma[i]];
  pout[i] = pin[sigma[i]];
}

// sorted coordinates, and the inverse permutation (input index -> sorted
// position) that the final reduction gathers through
__global__ void k_gather_xyz(const double *__restrict__ xyz, const int32_t *__restrict__ perm,
                             int64_t n, double *__restrict__ out, int32_t *__restrict__ iperm) {
  int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  int64_t j = perm[i];
  out[3 * i] = xyz[3 * j];
  out[3 * i + 1] = xyz[3 * j + 1];
  out[3 * i + 2] = xyz[3 * j + 2];
  iperm[j] = (int32_t)i;
}

// --------------------------------------------------------------- octree
__device__ __forceinline__ int32_t lower_bound_digit(const uint64_t *keys, int32_t f, int32_t e,
                                                     int shift, uint32_t o) {
  // first i in [f, e) with digit(i) >= o; digits are non-decreasing in the range
  while (f < e) {
    int32_t m = f + ((e - f) >> 1);
    if (((keys[m] >> shift) & 7u) < o) f = m + 1;
    else e = m;
  }
  return f;
}

// One warp per box of the level: lanes 0-7 find the 8 child boundaries (first
// key whose next 3-bit digit is >= o + 1) with independent binary searches,
// so the dependent-load chain of a box is one search deep, not eight.  The
// boundaries are kept for k_split_make.
__global__ void k_split_count(int level, int32_t b0, int32_t nbl, const int32_t *__restrict__ first,
                              const int32_t *__restrict__ count, const uint64_t *__restrict__ keys,
                              int leaf_size, int max_depth, int32_t *__restrict__ nchild,
                              int32_t *__restrict__ bnd) {
  const int lane = threadIdx.x & 31;
  const int32_t t = blockIdx.x * (kT / 32) + (threadIdx.x >> 5);
  if (t >= nbl) return;  // whole warp
  const int32_t b = b0 + t;
  const int32_t c = count[b];
  if (c <= leaf_size || level >= max_depth) {
    if (lane == 0) nchild[t] = 0;
    return;
  }
  const int shift = 3 * (kMaxDepth - (level + 1));
  const int32_t f = first[b], e = f + c;
  const int32_t s1 = lane < 8 ? lower_bound_digit(keys, f, e, shift, (uint32_t)lane + 1) : e;
  int32_t s0 = __shfl_up_sync(0xffffffffu, s1, 1);
  if (lane == 0) s0 = f;
  const unsigned nonempty = __ballot_sync(0xffffffffu, lane < 8 && s1 > s0);
  if (lane < 8) bnd[(int64_t)t * 8 + lane] = s1;
  if (lane == 0) nchild[t] = __popc(nonempty);
}

__global__ void k_split_make(int level, int32_t b0, int32_t nbl, int32_t child0,
                             const int32_t *__restrict__ nchild, const int32_t *__restrict__ coff,
                             const int32_t *__restrict__ bnd, int32_t *first, int32_t *count,
                             uint64_t *bkey, int32_t *blevel, int32_t *parent, int32_t *child,
                             int32_t *bnchild, int32_t *bprob) {
  int32_t t = blockIdx.x * kT + threadIdx.x;
  if (t >= nbl) return;
  int32_t b = b0 + t;
  int32_t k = nchild[t];
  bnchild[b] = k;
  if (k == 0) {
    child[b] = -1;
    return;
  }
  int32_t c = child0 + coff[t];
  child[b] = c;
  int32_t s = first[b];
  uint64_t pk = bkey[b];
  for (uint32_t o = 0; o < 8; ++o) {
    const int32_t s1 = bnd[(int64_t)t * 8 + o];
    if (s1 > s) {
      first[c] = s;
      count[c] = s1 - s;
      bkey[c] = (pk << 3) | o;
      blevel[c] = level + 1;
      parent[c] = b;
      bprob[c] = bprob[b];
      ++c;
    }
    s = s1;
  }
}

__global__ void k_box_geo(int64_t nb, const uint64_t *__restrict__ bkey,
                          const int32_t *__restrict__ blevel, BoxGeo *__restrict__ geo) {
  int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b >= nb) return;
  uint64_t k = bkey[b];
  BoxGeo g;
  g.ix = (int32_t)compact3(k);
  g.iy = (int32_t)compact3(k >> 1);
  g.iz = (int32_t)compact3(k >> 2);
  g.level = blevel[b];
  geo[b] = g;
}

__global__ void k_box_side(int64_t nb, const int32_t *__restrict__ blevel,
                           const int32_t *__restrict__ bprob, const double *__restrict__ geom,
                           double *__restrict__ side) {
  int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b >= nb) return;
  side[b] = box_side(geom[8 * bprob[b] + 3], blevel[b]);
}

__global__ void k_flag(int64_t n, const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                       int mode, int32_t *__restrict__ flag) {
  // mode 0: flag = (a[i] == 0)     (leaf: no children)
  // mode 1: flag = (a[i+1] > a[i]) (non-empty CSR row)
  // mode 2: flag = (b[i] == 0 && a[i+1] > a[i])
  int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  int32_t f;
  if (mode == 0) f = a[i] == 0;
  else if (mode == 1) f = a[i + 1] > a[i];
  else f = (b[i] == 0) && (a[i + 1] > a[i]);
  flag[i] = f;
}

__global__ void k_slot_of(int64_t nsel, const int32_t *__restrict__ sel, int32_t *__restrict__ slot) {
  int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (j < nsel) slot[sel[j]] = (int32_t)j;
}

__global__ void k_compact(int64_t n, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                          int32_t *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) out[pos[i]] = (int32_t)i;
}

// one warp per leaf (8 leaves per CTA): leaf-local coordinates x - c_leaf in
// FP64 and FP32
constexpr int kLeafWarps = 8;
__global__ void k_leaf_points(int64_t nleaves, const int32_t *__restrict__ leaves,
                              const BoxGeo *__restrict__ geo, const int32_t *__restrict__ first,
                              const int32_t *__restrict__ count, const double *__restrict__ xyz,
                              const int32_t *__restrict__ bprob, const double *__restrict__ pgeom,
                              const double *__restrict__ side, Dbl4 *__restrict__ pl64,
                              float4 *__restrict__ pl32) {
  const int64_t w = (int64_t)blockIdx.x * kLeafWarps + (threadIdx.x >> 5);
  if (w >= nleaves) return;
  const int lane = threadIdx.x & 31;
  int32_t b = leaves[w];
  BoxGeo g = geo[b];
  const double *lo = pgeom + 8 * bprob[b];
  double a = side[b];
  double cx = lo[0] + ((double)g.ix + 0.5) * a, cy = lo[1] + ((double)g.iy + 0.5) * a,
         cz = lo[2] + ((double)g.iz + 0.5) * a;
  int32_t f = first[b], c = count[b];
  for (int32_t i = f + lane; i < f + c; i += 32) {
    double x = xyz[3 * (int64_t)i] - cx, y = xyz[3 * (int64_t)i + 1] - cy,
           z = xyz[3 * (int64_t)i + 2] - cz;
    pl64[i] = make_dbl4(x, y, z, 0.0);
    pl32[i] = make_float4((float)x, (float)y, (float)z, 0.f);
  }
}

// ------------------------------------------------------------ adjacency
__device__ __forceinline__ bool adjacent(const BoxGeo &A, const BoxGeo &B) {
  int sa = kMaxDepth - A.level, sb = kMaxDepth - B.level;
  int64_t alo, ahi, blo, bhi;
  alo = (int64_t)A.ix << sa; ahi = ((int64_t)A.ix + 1) << sa;
  blo = (int64_t)B.ix << sb; bhi = ((int64_t)B.ix + 1) << sb;
  if (alo > bhi || blo > ahi) return false;
  alo = (int64_t)A.iy << sa; ahi = ((int64_t)A.iy + 1) << sa;
  blo = (int64_t)B.iy << sb; bhi = ((int64_t)B.iy + 1) << sb;
  if (alo > bhi || blo > ahi) return false;
  alo = (int64_t)A.iz << sa; ahi = ((int64_t)A.iz + 1) << sa;
  blo = (int64_t)B.iz << sb; bhi = ((int64_t)B.iz + 1) << sb;
  if (alo > bhi || blo > ahi) return false;
  return true;
}

// colleagues: same-level boxes adjacent to B (excluding B), ascending
__global__ void k_colleagues(int64_t nb, const BoxGeo *__restrict__ geo,
                             const uint64_t *__restrict__ bkey, const int32_t *__restrict__ bprob,
                             const int32_t *__restrict__ loff, int32_t *__restrict__ col,
                             int32_t *__restrict__ ncol) {
  int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b >= nb) return;
  BoxGeo g = geo[b];
  const int32_t pb = bprob[b];  // boxes of a level are ordered by (problem, key)
  int32_t found[26];
  int k = 0;
  if (g.level > 0) {
    const int32_t lo = loff[g.level], hi = loff[g.level + 1];
    const int32_t lim = 1 << g.level;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          int32_t x = g.ix + dx, y = g.iy + dy, z = g.iz + dz;
          if (x < 0 || y < 0 || z < 0 || x >= lim || y >= lim || z >= lim) continue;
          uint64_t key = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
          int32_t f = lo, e = hi;
          while (f < e) {
            int32_t m = f + ((e - f) >> 1);
            if (bprob[m] < pb || (bprob[m] == pb && bkey[m] < key)) f = m + 1;
            else e = m;
          }
          if (f < hi && bprob[f] == pb && bkey[f] == key) {
            int j = k++;  // insertion sort
            while (j > 0 && found[j - 1] > f) {
              found[j] = found[j - 1];
              --j;
            }
            found[j] = f;
          }
        }
  }
  for (int j = 0; j < 26; ++j) col[26 * b + j] = j < k ? found[j] : -1;
  ncol[b] = k;
}

// V(B), level >= 2: children of colleagues of parent(B) not adjacent to B
template <bool kFill>
__global__ void k_vlist(int64_t nb, const BoxGeo *__restrict__ geo, const int32_t *__restrict__ parent,
                        const int32_t *__restrict__ child, const int32_t *__restrict__ nchild,
                        const int32_t *__restrict__ col, const int32_t *__restrict__ ncol,
                        int32_t *__restrict__ cnt, const int32_t *__restrict__ off,
                        int32_t *__restrict__ idx) {
  int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b >= nb) return;
  BoxGeo g = geo[b];
  int32_t k = 0;
  int32_t o = kFill ? off[b] : 0;
  if (g.level >= 2) {
    int32_t P = parent[b];
    for (int j = 0; j < ncol[P]; ++j) {
      int32_t C = col[26 * (int64_t)P + j];
      int32_t c0 = child[C], c1 = c0 + nchild[C];
      for (int32_t A = c0; A < c1; ++A) {
        if (!adjacent(geo[A], g)) {
          if (kFill) idx[o + k] = A;
          ++k;
        }
      }
    }
  }
  if (!kFill) cnt[b] = k;
}

// CA(B): leaves with level <= level(B), adjacent to B, other than B.  They are
// the leaf colleagues of B's ancestors (and of B) that touch B; ascending.
template <bool kFill>
__global__ void k_calist(int64_t nb, const BoxGeo *__restrict__ geo, const int32_t *__restrict__ parent,
                         const int32_t *__restrict__ nchild, const int32_t *__restrict__ col,
                         const int32_t *__restrict__ ncol, int32_t *__restrict__ cnt,
                         const int32_t *__restrict__ off, int32_t *__restrict__ idx) {
  int64_t b = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (b >= nb) return;
  BoxGeo g = geo[b];
  int32_t chain[kMaxDepth + 1];
  int32_t Q = (int32_t)b;
  for (int l = g.level; l >= 0; --l) {
    chain[l] = Q;
    Q = parent[Q];
  }
  int32_t k = 0;
  int32_t o = kFill ? off[b] : 0;
  for (int l = 1; l <= g.level; ++l) {
    int32_t A = chain[l];
    for (int j = 0; j < ncol[A]; ++j) {
      int32_t C = col[26 * (int64_t)A + j];
      if (nchild[C] == 0 && adjacent(geo[C], g)) {
        if (kFill) idx[o + k] = C;
        ++k;
      }
    }
  }
  if (!kFill) cnt[b] = k;
}

// U pairs of leaf B: (B,B), (B,A) for A in CA(B), and (A,B) for the coarser
// A in CA(B) (finer adjacent leaves find B in their own CA lists).

// X(C) = { A in CA(parent(C)) : A not adjacent to C }
template <bool kFill>
__global__ void k_xlist(int64_t nb, const BoxGeo *__restrict__ geo, const int32_t *__restrict__ parent,
                        const int32_t *__restrict__ caoff, const int32_t *__restrict__ caidx,
                        int32_t *__restrict__ cnt, const int32_t *__restrict__ off,
                        int32_t *__restrict__ idx) {
  int64_t C = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (C >= nb) return;
  BoxGeo g = geo[C];
  int32_t k = 0;
  int32_t o = kFill ? off[C] : 0;
  if (g.level >= 2) {
    int32_t P = parent[C];
    for (int32_t e = caoff[P]; e < caoff[P + 1]; ++e) {
      int32_t A = caidx[e];
      if (!adjacent(geo[A], g)) {
        if (kFill) idx[o + k] = A;
        ++k;
      }
    }
  }
  if (!kFill) cnt[C] = k;
}

// W pairs from X: (A, C) for every A in X(C)
// pending boxes of the descent: at most the 26 colleagues plus 8 children per
// level of depth (194), so the overflow check below never fires
constexpr int kUWStack = 256;

// U and W of one leaf B, without a global sort.  U(B) is the leaf itself,
// its coarser-or-equal adjacent leaves CA(B) (already in box order), and the
// finer leaves adjacent to it.  Those lie inside B's colleagues, and so do
// the boxes of W(B) (not adjacent to B, parent adjacent).  One descent from
// the colleagues finds both: a child of a box adjacent to B goes to U if it
// is an adjacent leaf, to W if it is not adjacent, and is descended into if
// it is adjacent with children.  Box numbers are level-major, so the finer U
// entries all follow the coarser-or-equal ones; each finer run and each W
// run is sorted in place.  Count pass (kFill = false) and fill pass.
template <bool kFill>
__global__ void k_uwlist(int64_t nl, const int32_t *__restrict__ leaves,
                         const BoxGeo *__restrict__ geo, const int32_t *__restrict__ child,
                         const int32_t *__restrict__ nchild, const int32_t *__restrict__ col,
                         const int32_t *__restrict__ ncol, const int32_t *__restrict__ caoff,
                         const int32_t *__restrict__ caidx, int32_t *__restrict__ ucnt,
                         int32_t *__restrict__ wcnt, const int32_t *__restrict__ uoff,
                         int32_t *__restrict__ uidx, const int32_t *__restrict__ woff,
                         int32_t *__restrict__ widx, int *__restrict__ err) {
  const int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (t >= nl) return;
  const int32_t B = leaves[t];
  const BoxGeo gB = geo[B];
  const int32_t c0 = caoff[B], c1 = caoff[B + 1];
  int64_t ou = 0, ow = 0;
  if (kFill) {
    ou = uoff[B];
    ow = woff[B];
    int64_t k = ou;  // CA(B) with B merged in at its place
    bool placed = false;
    for (int32_t e = c0; e < c1; ++e) {
      const int32_t A = caidx[e];
      if (!placed && A > B) {
        uidx[k++] = B;
        placed = true;
      }
      uidx[k++] = A;
    }
    if (!placed) uidx[k++] = B;
  }
  int32_t ku = (c1 - c0) + 1, kw = 0;
  const int32_t kfine = ku;
  int32_t stack[kUWStack];
  int sp = 0;
  bool overflow = false;
  for (int j = 0; j < ncol[B]; ++j) {
    const int32_t C = col[26 * (int64_t)B + j];
    if (nchild[C] > 0) stack[sp++] = C;  // 26 <= kUWStack
  }
  while (sp > 0 && !overflow) {
    const int32_t D = stack[--sp];
    const int32_t e0 = child[D], e1 = e0 + nchild[D];
    for (int32_t E = e0; E < e1; ++E) {
      const BoxGeo gE = geo[E];
      if (adjacent(gE, gB)) {
        if (nchild[E] == 0) {
          if (kFill) uidx[ou + ku] = E;
          ++ku;
        } else if (sp < kUWStack) {
          stack[sp++] = E;
        } else {
          overflow = true;
        }
      } else {
        if (kFill) widx[ow + kw] = E;
        ++kw;
      }
    }
  }
  if (overflow) {
    atomicExch(err, 1);
    return;
  }
  if (!kFill) {
    ucnt[B] = ku;
    wcnt[B] = kw;
  } else {
    sort_run(uidx + ou + kfine, ku - kfine);
    sort_run(widx + ow, kw);
  }
}


// CSR rows from (row << 32 | col) keys sorted ascending

// M2L ordering key: (level, parity) class of every box of level >= 2
__global__ void k_m2l_class(int64_t b0, int64_t nb, const BoxGeo *__restrict__ geo,
                            uint64_t *__restrict__ key, int32_t *__restrict__ val,
                            int32_t *__restrict__ hist) {
  int64_t t = (int64_t)blockIdx.x * kT + threadIdx.x;
  if (t >= nb - b0) return;
  int64_t b = b0 + t;
  BoxGeo g = geo[b];
  int cls = g.level * 8 + (g.ix & 1) + 2 * (g.iy & 1) + 4 * (g.iz & 1);
  key[t] = (uint64_t)cls;
  val[t] = (int32_t)b;
  atomicAdd(&hist[cls], 1);
}

inline int grid(int64_t n) { return n > 0 ? ceil_div(n, kT) : 1; }

int bits_for(int64_t v) {
  int b = 1;
  while ((int64_t(1) << b) <= v) ++b;
  return b;
}

// CSR row offsets (nb+1) from per-row counts (nb); returns the total
int64_t counts_to_offsets(fmm_plan_impl &P, const int32_t *cnt, DBuf<int32_t> &off, int64_t nrows) {
  off.resize(nrows + 1, P.stream);
  scan_exclusive(cnt, off.p, nrows, off.p + nrows, P.s_scan, P.stream);
  return read_scalar(off.p + nrows, P.stream);
}

// the same without reading the total back (off[nrows] holds it on the device)
void counts_to_offsets_async(fmm_plan_impl &P, const int32_t *cnt, DBuf<int32_t> &off,
                             int64_t nrows) {
  off.resize(nrows + 1, P.stream);
  scan_exclusive(cnt, off.p, nrows, off.p + nrows, P.s_scan, P.stream);
}

int64_t compact(fmm_plan_impl &P, int64_t n, const int32_t *flag, DBuf<int32_t> &out) {
  cudaStream_t s = P.stream;
  P.s_i32c.resize(n + 1, s);
  scan_exclusive(flag, P.s_i32c.p, n, P.s_i32c.p + n, P.s_scan, s);
  int64_t m = read_scalar(P.s_i32c.p + n, s);
  out.resize(m > 0 ? m : 1, s);
  k_compact<<<grid(n), kT, 0, s>>>(n, flag, P.s_i32c.p, out.p);
  FMM_LAUNCH_CHECK();
  return m;
}


// ---- small W/X leaf pairs to the near field (fmm_opts.wx_direct)
// A pair of leaves (B, A) with A in W(B) and A holding at most T points moves
// to the near field in both directions: A joins U(B) and B joins U(A); A
// leaves W(B) and B leaves X(A).  For box b: its W entries that are such
// leaves move to U(b); its X entries C (C a leaf with b in W(C)) all move when
// b is a leaf of at most T points, none otherwise.  The operator stays
// symmetric; U rows are re-sorted.
__global__ void k_wx_direct_count(int64_t nb, int T, const int32_t *__restrict__ nchild,
                                  const int32_t *__restrict__ count, const int32_t *__restrict__ uoff,
                                  const int32_t *__restrict__ woff, const int32_t *__restrict__ widx,
                                  const int32_t *__restrict__ xoff, int32_t *__restrict__ ucnt,
                                  int32_t *__restrict__ wcnt, int32_t *__restrict__ xcnt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const bool leaf = nchild[b] == 0;
  int32_t moved = 0, kept = 0;
  for (int32_t e = woff[b]; e < woff[b + 1]; ++e) {
    const int32_t A = widx[e];
    if (leaf && nchild[A] == 0 && count[A] <= T)
      ++moved;
    else
      ++kept;
  }
  const int32_t nx = xoff[b + 1] - xoff[b];
  const bool xmove = leaf && count[b] <= T;
  ucnt[b] = uoff[b + 1] - uoff[b] + moved + (xmove ? nx : 0);
  wcnt[b] = kept;
  xcnt[b] = xmove ? 0 : nx;
}

// The new U row of b merges three rows that are already sorted: its U row,
// the W entries that move and (when they all move) its X row; the lists are
// disjoint, so the merge never meets a box twice.
__global__ void k_wx_direct_fill(int64_t nb, int T, const int32_t *__restrict__ nchild,
                                 const int32_t *__restrict__ count, const int32_t *__restrict__ uoff,
                                 const int32_t *__restrict__ uidx, const int32_t *__restrict__ woff,
                                 const int32_t *__restrict__ widx, const int32_t *__restrict__ xoff,
                                 const int32_t *__restrict__ xidx, const int32_t *__restrict__ nuoff,
                                 int32_t *__restrict__ nuidx, const int32_t *__restrict__ nwoff,
                                 int32_t *__restrict__ nwidx, const int32_t *__restrict__ nxoff,
                                 int32_t *__restrict__ nxidx) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const bool leaf = nchild[b] == 0;
  const bool xmove = leaf && count[b] <= T;
  auto moves = [&](int32_t A) { return leaf && nchild[A] == 0 && count[A] <= T; };
  int32_t *u = nuidx + nuoff[b], *w = nwidx + nwoff[b], *x = nxidx + nxoff[b];
  int32_t kw = 0, kx = 0;
  for (int32_t e = woff[b]; e < woff[b + 1]; ++e)
    if (!moves(widx[e])) w[kw++] = widx[e];
  if (!xmove)
    for (int32_t e = xoff[b]; e < xoff[b + 1]; ++e) x[kx++] = xidx[e];
  int32_t iu = uoff[b], iw = woff[b], ix = xoff[b];
  const int32_t eu = uoff[b + 1], ew = woff[b + 1], ex = xmove ? xoff[b + 1] : xoff[b];
  while (iw < ew && !moves(widx[iw])) ++iw;
  int32_t k = 0;
  while (true) {
    const int32_t cu = iu < eu ? uidx[iu] : INT32_MAX, cw = iw < ew ? widx[iw] : INT32_MAX,
                  cx = ix < ex ? xidx[ix] : INT32_MAX;
    const int32_t m = min(cu, min(cw, cx));
    if (m == INT32_MAX) break;
    u[k++] = m;
    if (m == cu) {
      ++iu;
    } else if (m == cw) {
      ++iw;
      while (iw < ew && !moves(widx[iw])) ++iw;
    } else {
      ++ix;
    }
  }
}

void direct_wx_pairs(fmm_plan_impl &P, int T) {
  cudaStream_t s = P.stream;
  const int64_t nb = P.nboxes;
  DBuf<int32_t> &ucnt = P.s_i32a, &wcnt = P.s_i32d, &xcnt = P.s_i32c;
  ucnt.resize(nb, s);
  wcnt.resize(nb, s);
  xcnt.resize(nb, s);
  k_wx_direct_count<<<grid(nb), kT, 0, s>>>(nb, T, P.box_nchild.p, P.box_count.p, P.u_off.p,
                                             P.w_off.p, P.w_idx.p, P.x_off.p, ucnt.p, wcnt.p, xcnt.p);
  FMM_LAUNCH_CHECK();
  DBuf<int32_t> uo, ui, wo, wi, xo, xi;
  counts_to_offsets_async(P, ucnt.p, uo, nb);
  counts_to_offsets_async(P, wcnt.p, wo, nb);
  counts_to_offsets_async(P, xcnt.p, xo, nb);
  int32_t h[3];
  FMM_CUDA(cudaMemcpyAsync(&h[0], uo.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaMemcpyAsync(&h[1], wo.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaMemcpyAsync(&h[2], xo.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  ui.resize(h[0] > 0 ? h[0] : 1, s);
  wi.resize(h[1] > 0 ? h[1] : 1, s);
  xi.resize(h[2] > 0 ? h[2] : 1, s);
  k_wx_direct_fill<<<grid(nb), kT, 0, s>>>(nb, T, P.box_nchild.p, P.box_count.p, P.u_off.p,
                                            P.u_idx.p, P.w_off.p, P.w_idx.p, P.x_off.p, P.x_idx.p,
                                            uo.p, ui.p, wo.p, wi.p, xo.p, xi.p);
  FMM_LAUNCH_CHECK();
  std::swap(P.u_off, uo);
  std::swap(P.u_idx, ui);
  std::swap(P.w_off, wo);
  std::swap(P.w_idx, wi);
  std::swap(P.x_off, xo);
  std::swap(P.x_idx, xi);
  uo.release();
  ui.release();
  wo.release();
  wi.release();
  xo.release();
  xi.release();
  P.nu = h[0];
  P.nw = h[1];
  P.nx = h[2];
}

}  // namespace

// Rotated M2L: on request (m2l_path 3), and by default in FP64 up to
// kRotMaxOrder, where it runs 1.7-2x faster than the dense FP64 operator
// (FP64 multiply-adds are scarce on this GPU); the FP32 paths keep the
// dense operators (tensor cores up to order 10, CUDA cores above).
bool uses_rotation(const fmm_plan_impl &P) {
  if (P.dual || P.order > kRotMaxOrder) return false;
  return P.m2l_path == 3 || (P.m2l_path == 0 && P.precision == FMM_FP64);
}

// M2L tiles: boxes of level >= 2 grouped by (level, octant parity), and for
// the mixed-precision paths the per-tile source tables
void build_m2l_tiles(fmm_plan_impl &P) {
  cudaStream_t s = P.stream;
  const int64_t nb = P.nboxes;
  P.m2l_tc = P.precision == FMM_MIXED && P.order <= kM2LStagedMaxOrder && P.m2l_path != 1 &&
             P.m2l_path != 3;
  P.m2l_rot = uses_rotation(P);
  P.m2l_tile_size = P.m2l_tc ? kM2LTensorTile : m2l_tile_size(P.order, P.precision);
  int64_t b2 = P.nlevels > 2 ? P.level_off[2] : nb;
  int64_t n2 = nb - b2;
  if (n2 > 0) {
    const int ncls = 8 * (kMaxDepth + 1);
    P.s_hist.resize(ncls, s);
    FMM_CUDA(cudaMemsetAsync(P.s_hist.p, 0, sizeof(int32_t) * ncls, s));
    P.s_u64a.resize(n2, s);
    P.m2l_order.resize(n2, s);
    k_m2l_class<<<grid(n2), kT, 0, s>>>(b2, nb, P.box_geo.p, P.s_u64a.p, P.m2l_order.p, P.s_hist.p);
    FMM_LAUNCH_CHECK();
    std::vector<int32_t> h(ncls);
    FMM_CUDA(cudaMemcpyAsync(h.data(), P.s_hist.p, sizeof(int32_t) * ncls, cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    radix_sort(P.s_u64a, P.m2l_order, P.s_u64b, P.s_i32a, n2, {0}, P.s_hist, P.s_scan, s);
    std::vector<M2LTile> tiles;
    int32_t o = 0, T = P.m2l_tile_size;
    for (int c = 0; c < ncls; ++c) {
      for (int32_t t = 0; t < h[c]; t += T) tiles.push_back({o + t, std::min(T, h[c] - t), c & 7, 0});
      o += h[c];
    }
    P.nm2l_tiles = (int64_t)tiles.size();
    P.m2l_tiles.resize(tiles.size(), s);
    FMM_CUDA(cudaMemcpyAsync(P.m2l_tiles.p, tiles.data(), sizeof(M2LTile) * tiles.size(),
                             cudaMemcpyHostToDevice, s));
    FMM_CUDA(cudaStreamSynchronize(s));  // `tiles` is a host temporary
    if ((P.precision == FMM_MIXED && P.order <= kM2LStagedMaxOrder) || P.m2l_rot)
      build_m2l_tables(P);
  }
}

void build_vlists(fmm_plan_impl &P) {
  cudaStream_t s = P.stream;
  const int64_t nb = P.nboxes;
  P.v_built = true;
  P.nv = 0;
  if (nb == 0) return;
  if (P.dual) return;  // a dual-tree plan keeps its M2L pairs in V
  P.s_i32a.resize(nb, s);
  k_vlist<false><<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_parent.p, P.box_child.p,
                                          P.box_nchild.p, P.colleagues.p, P.ncolleagues.p,
                                          P.s_i32a.p, nullptr, nullptr);
  FMM_LAUNCH_CHECK();
  P.nv = counts_to_offsets(P, P.s_i32a.p, P.v_off, nb);
  P.v_idx.resize(P.nv > 0 ? P.nv : 1, s);
  k_vlist<true><<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_parent.p, P.box_child.p,
                                         P.box_nchild.p, P.colleagues.p, P.ncolleagues.p, nullptr,
                                         P.v_off.p, P.v_idx.p);
  FMM_LAUNCH_CHECK();
}

int32_t read_scalar(const int32_t *d, cudaStream_t s) {
  int32_t h = 0;
  FMM_CUDA(cudaMemcpyAsync(&h, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  return h;
}

void morton_keys_raw(const double *d_xyz, int64_t n, double *partial, double *geom, uint64_t *keys,
                     int32_t *perm, cudaStream_t s) {
  if (n <= 0) return;
  int nbb = std::min(ceil_div(n, kT * 8), 1024);
  k_bbox_partial<<<nbb, kT, 0, s>>>(d_xyz, n, partial);
  FMM_LAUNCH_CHECK();
  k_bbox_final<<<1, kT, 0, s>>>(partial, nbb, geom);
  FMM_LAUNCH_CHECK();
  k_morton<<<grid(n), kT, 0, s>>>(d_xyz, n, geom, nullptr, 1, keys, perm);
  FMM_LAUNCH_CHECK();
}

void set_points(fmm_plan_impl &P, const double *d_xyz) {
  cudaStream_t s = P.stream;
  int64_t n = P.n;
  if (n == 0) return;
  P.iperm.resize(n, s);
  k_gather_xyz<<<grid(n), kT, 0, s>>>(d_xyz, P.perm.p, n, P.xyz_sorted.p, P.iperm.p);
  FMM_LAUNCH_CHECK();
  if (P.nleaves > 0)
    k_leaf_points<<<(unsigned)ceil_div(P.nleaves, (int64_t)kLeafWarps), 32 * kLeafWarps, 0, s>>>(
        P.nleaves, P.leaves.p, P.box_geo.p, P.box_first.p, P.box_count.p, P.xyz_sorted.p,
        P.box_prob.p, P.prob_geom.p, P.box_side.p, P.pl64.p, P.pl32.p);
  FMM_LAUNCH_CHECK();
}

void build_tree(fmm_plan_impl &P, const double *d_xyz, int64_t n) {
  cudaStream_t s = P.stream;
  drop_graph(P);  // a captured graph refers to the old layout
  P.p2p_meta_ok = false;
  P.oct_ok = false;
  P.n = n;
  P.nboxes = 0;
  P.nlevels = 0;
  P.level_off.assign(1, 0);
  P.nu = P.nv = P.nw = P.nx = 0;
  P.v_built = true;
  P.nleaves = P.nxboxes = P.nwleaves = P.nm2l_tiles = 0;
  if (n == 0) return;
  std::unique_ptr<PassScope> scope(new PassScope(P, kPassSort));

  // ---- root cube(s)
  const int B = P.nproblems;
  if ((int64_t)P.prob_off_h.size() != B + 1 || P.prob_off_h[B] != n) P.prob_off_h = {0, n};
  P.prob_geom.resize((size_t)8 * B, s);
  if (B == 1) {
    int nbb = std::min(ceil_div(n, kT * 8), 1024);
    P.partial.resize((size_t)7 * nbb, s);
    k_bbox_partial<<<nbb, kT, 0, s>>>(d_xyz, n, P.partial.p);
    FMM_LAUNCH_CHECK();
    k_bbox_final<<<1, kT, 0, s>>>(P.partial.p, nbb, P.prob_geom.p);
    FMM_LAUNCH_CHECK();
  } else {
    P.prob_off.resize(B + 1, s);
    FMM_CUDA(cudaMemcpyAsync(P.prob_off.p, P.prob_off_h.data(), sizeof(int64_t) * (B + 1),
                             cudaMemcpyHostToDevice, s));
    k_bbox_problems<<<B, kT, 0, s>>>(d_xyz, P.prob_off.p, P.prob_geom.p);
    FMM_LAUNCH_CHECK();
  }
  P.prob_geom_h.resize((size_t)8 * B);
  FMM_CUDA(cudaMemcpyAsync(P.prob_geom_h.data(), P.prob_geom.p, sizeof(double) * 8 * B,
                           cudaMemcpyDeviceToHost, s));
  FMM_CUDA(cudaStreamSynchronize(s));
  for (int b = 0; b < B; ++b)
    if (P.prob_geom_h[8 * b + 4] != 0.0)
      throw Error(FMM_ERR_NONFINITE_INPUT, "a coordinate is NaN or infinite");
  P.lo[0] = P.prob_geom_h[0];
  P.lo[1] = P.prob_geom_h[1];
  P.lo[2] = P.prob_geom_h[2];
  P.D = P.prob_geom_h[3];

  // ---- keys and stable sort (by key; for a batch, then stably by problem)
  P.keys.resize(n, s);
  P.perm.resize(n, s);
  k_morton<<<grid(n), kT, 0, s>>>(d_xyz, n, P.prob_geom.p, B > 1 ? P.prob_off.p : nullptr, B,
                                   P.keys.p, P.perm.p);
  FMM_LAUNCH_CHECK();
  radix_sort(P.keys, P.perm, P.keys_tmp, P.perm_tmp, n, digit_shifts(0, 3 * kMaxDepth), P.s_hist,
             P.s_scan, s);
  if (B > 1) {
    P.s_u64a.resize(n, s);
    P.s_i32a.resize(n, s);
    k_problem_keys<<<grid(n), kT, 0, s>>>(n, P.perm.p, P.prob_off.p, B, P.s_u64a.p, P.s_i32a.p);
    FMM_LAUNCH_CHECK();
    radix_sort(P.s_u64a, P.s_i32a, P.s_u64b, P.s_i32b, n, digit_shifts(0, bits_for(B)), P.s_hist,
               P.s_scan, s);
    k_apply_perm<<<grid(n), kT, 0, s>>>(n, P.s_i32a.p, P.keys.p, P.perm.p, P.keys_tmp.p,
                                         P.perm_tmp.p);
    FMM_LAUNCH_CHECK();
    std::swap(P.keys, P.keys_tmp);
    std::swap(P.perm, P.perm_tmp);
  }
  P.xyz_sorted.resize(3 * n, s);
  P.iperm.resize(n, s);
  k_gather_xyz<<<grid(n), kT, 0, s>>>(d_xyz, P.perm.p, n, P.xyz_sorted.p, P.iperm.p);
  FMM_LAUNCH_CHECK();

  // ---- boxes, level by level; level 0 holds one root per non-empty problem
  scope.reset(new PassScope(P, kPassBoxes));
  size_t cap0 = std::max<size_t>(1024 + B, 2 * (size_t)n / (size_t)P.leaf_size + 64 + B);
  auto grow_boxes = [&](size_t need, size_t keep) {
    P.box_key.grow(std::max(need, cap0), keep, s);
    P.box_level.grow(std::max(need, cap0), keep, s);
    P.box_first.grow(std::max(need, cap0), keep, s);
    P.box_count.grow(std::max(need, cap0), keep, s);
    P.box_parent.grow(std::max(need, cap0), keep, s);
    P.box_child.grow(std::max(need, cap0), keep, s);
    P.box_nchild.grow(std::max(need, cap0), keep, s);
    P.box_prob.grow(std::max(need, cap0), keep, s);
  };
  std::vector<uint64_t> rk;
  std::vector<int32_t> rz, rf, rc, rm, rp;
  for (int b = 0; b < B; ++b) {
    const int64_t c = P.prob_off_h[b + 1] - P.prob_off_h[b];
    if (c == 0) continue;
    rk.push_back(0);
    rz.push_back(0);
    rf.push_back((int32_t)P.prob_off_h[b]);
    rc.push_back((int32_t)c);
    rm.push_back(-1);
    rp.push_back(b);
  }
  const int64_t nroots = (int64_t)rk.size();
  grow_boxes(nroots, 0);
  FMM_CUDA(cudaMemcpyAsync(P.box_key.p, rk.data(), 8 * nroots, cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.box_level.p, rz.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.box_first.p, rf.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.box_count.p, rc.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.box_parent.p, rm.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaMemcpyAsync(P.box_prob.p, rp.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  FMM_CUDA(cudaStreamSynchronize(s));  // the host vectors above are temporaries
  P.level_off = {0, (int32_t)nroots};
  int64_t nb = nroots;
  for (int l = 0;; ++l) {
    int32_t b0 = P.level_off[l], nbl = P.level_off[l + 1] - b0;
    P.s_i32a.resize(nbl + 1, s);
    P.s_i32b.resize(nbl + 1, s);
    P.s_i32c.resize((size_t)nbl * 8, s);  // child boundaries, 8 per box
    k_split_count<<<ceil_div((int64_t)nbl, (int64_t)(kT / 32)), kT, 0, s>>>(
        l, b0, nbl, P.box_first.p, P.box_count.p, P.keys.p, P.leaf_size, P.max_depth, P.s_i32a.p,
        P.s_i32c.p);
    FMM_LAUNCH_CHECK();
    scan_exclusive(P.s_i32a.p, P.s_i32b.p, nbl, P.s_i32b.p + nbl, P.s_scan, s);
    int32_t nnew = read_scalar(P.s_i32b.p + nbl, s);
    if (nnew > 0) grow_boxes(nb + nnew, nb);
    k_split_make<<<grid(nbl), kT, 0, s>>>(l, b0, nbl, (int32_t)nb, P.s_i32a.p, P.s_i32b.p,
                                           P.s_i32c.p, P.box_first.p, P.box_count.p, P.box_key.p,
                                           P.box_level.p, P.box_parent.p, P.box_child.p,
                                           P.box_nchild.p, P.box_prob.p);
    FMM_LAUNCH_CHECK();
    if (nnew == 0) break;
    nb += nnew;
    P.level_off.push_back((int32_t)nb);
  }
  P.nboxes = nb;
  P.nlevels = (int)P.level_off.size() - 1;

  P.box_geo.resize(nb, s);
  k_box_geo<<<grid(nb), kT, 0, s>>>(nb, P.box_key.p, P.box_level.p, P.box_geo.p);
  FMM_LAUNCH_CHECK();
  P.box_side.resize(nb, s);
  k_box_side<<<grid(nb), kT, 0, s>>>(nb, P.box_level.p, P.box_prob.p, P.prob_geom.p, P.box_side.p);
  FMM_LAUNCH_CHECK();

  // ---- leaves and leaf-local coordinates
  P.s_i32a.resize(nb, s);
  k_flag<<<grid(nb), kT, 0, s>>>(nb, P.box_nchild.p, nullptr, 0, P.s_i32a.p);
  FMM_LAUNCH_CHECK();
  P.nleaves = compact(P, nb, P.s_i32a.p, P.leaves);
  P.pl64.resize(n, s);
  P.pl32.resize(n, s);
  k_leaf_points<<<(unsigned)ceil_div(P.nleaves, (int64_t)kLeafWarps), 32 * kLeafWarps, 0, s>>>(
      P.nleaves, P.leaves.p, P.box_geo.p, P.box_first.p, P.box_count.p, P.xyz_sorted.p,
      P.box_prob.p, P.prob_geom.p, P.box_side.p, P.pl64.p, P.pl32.p);
  FMM_LAUNCH_CHECK();

  scope.reset(new PassScope(P, kPassLists));
  if (P.dual) {
    build_dual_lists(P);
    return;
  }

  // ---- colleagues
  DBuf<int32_t> &loff = P.s_i32b;
  loff.resize(P.level_off.size(), s);
  FMM_CUDA(cudaMemcpyAsync(loff.p, P.level_off.data(), sizeof(int32_t) * P.level_off.size(),
                           cudaMemcpyHostToDevice, s));
  P.colleagues.resize((size_t)26 * nb, s);
  P.ncolleagues.resize(nb, s);
  k_colleagues<<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_key.p, P.box_prob.p, loff.p,
                                        P.colleagues.p, P.ncolleagues.p);
  FMM_LAUNCH_CHECK();
  FMM_CUDA(cudaStreamSynchronize(s));  // level_off host vector must outlive the copy

  // ---- V lists: the mixed-precision M2L of orders <= kM2LStagedMaxOrder reads
  // its per-tile source table, built from the colleagues; the CSR is then
  // built only on request (fmm_plan_sizes / fmm_plan_export)
  P.v_built = false;
  const bool table_path =
      (P.precision == FMM_MIXED && P.order <= kM2LStagedMaxOrder) || uses_rotation(P);
  if (!table_path) build_vlists(P);

  // ---- coarser-or-equal adjacent leaves (CA)
  k_calist<false><<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_parent.p, P.box_nchild.p,
                                           P.colleagues.p, P.ncolleagues.p, P.s_i32a.p, nullptr,
                                           nullptr);
  FMM_LAUNCH_CHECK();
  // CA(B) holds distinct leaves no smaller than B that touch it, which do not
  // overlap: at most 26 (and X(C), a subset of CA(parent(C)), too), so both
  // are allocated at 26 entries per box without reading their totals back
  counts_to_offsets_async(P, P.s_i32a.p, P.ca_off, nb);
  P.ca_idx.resize((size_t)26 * std::max<int64_t>(nb, 1), s);
  k_calist<true><<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_parent.p, P.box_nchild.p,
                                          P.colleagues.p, P.ncolleagues.p, nullptr, P.ca_off.p,
                                          P.ca_idx.p);
  FMM_LAUNCH_CHECK();

  // ---- X lists (box C: the adjacent leaves of its parent's level or coarser
  // that are not adjacent to C)
  k_xlist<false><<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_parent.p, P.ca_off.p, P.ca_idx.p,
                                          P.s_i32a.p, nullptr, nullptr);
  FMM_LAUNCH_CHECK();
  counts_to_offsets_async(P, P.s_i32a.p, P.x_off, nb);
  P.x_idx.resize((size_t)26 * std::max<int64_t>(nb, 1), s);
  k_xlist<true><<<grid(nb), kT, 0, s>>>(nb, P.box_geo.p, P.box_parent.p, P.ca_off.p, P.ca_idx.p,
                                         nullptr, P.x_off.p, P.x_idx.p);
  FMM_LAUNCH_CHECK();

  // ---- U and W lists of the leaves (one descent per leaf, rows sorted in place)
  {
    const int64_t nl = P.nleaves;
    DBuf<int32_t> &ucnt = P.s_i32a, &wcnt = P.s_i32d;
    ucnt.resize(nb, s);
    wcnt.resize(nb, s);
    FMM_CUDA(cudaMemsetAsync(ucnt.p, 0, sizeof(int32_t) * nb, s));
    FMM_CUDA(cudaMemsetAsync(wcnt.p, 0, sizeof(int32_t) * nb, s));
    if (!P.dev_err.p) {
      P.dev_err.resize(1, s);
      FMM_CUDA(cudaMemsetAsync(P.dev_err.p, 0, sizeof(int), s));
    }
    k_uwlist<false><<<grid(nl), kT, 0, s>>>(nl, P.leaves.p, P.box_geo.p, P.box_child.p,
                                             P.box_nchild.p, P.colleagues.p, P.ncolleagues.p,
                                             P.ca_off.p, P.ca_idx.p, ucnt.p, wcnt.p, nullptr,
                                             nullptr, nullptr, nullptr, P.dev_err.p);
    FMM_LAUNCH_CHECK();
    counts_to_offsets_async(P, ucnt.p, P.u_off, nb);
    counts_to_offsets_async(P, wcnt.p, P.w_off, nb);
    {  // the X, U and W totals in one read-back
      int32_t h[3];
      FMM_CUDA(cudaMemcpyAsync(&h[0], P.x_off.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FMM_CUDA(cudaMemcpyAsync(&h[1], P.u_off.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FMM_CUDA(cudaMemcpyAsync(&h[2], P.w_off.p + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FMM_CUDA(cudaStreamSynchronize(s));
      P.nx = h[0];
      P.nu = h[1];
      P.nw = h[2];
    }
    P.u_idx.resize(P.nu > 0 ? P.nu : 1, s);
    P.w_idx.resize(P.nw > 0 ? P.nw : 1, s);
    k_uwlist<true><<<grid(nl), kT, 0, s>>>(nl, P.leaves.p, P.box_geo.p, P.box_child.p,
                                            P.box_nchild.p, P.colleagues.p, P.ncolleagues.p,
                                            P.ca_off.p, P.ca_idx.p, nullptr, nullptr, P.u_off.p,
                                            P.u_idx.p, P.w_off.p, P.w_idx.p, P.dev_err.p);
    FMM_LAUNCH_CHECK();
  }

  if (P.wx_direct_max > 0 && P.nw > 0) direct_wx_pairs(P, P.wx_direct_max);

  // ---- work lists for P2L and M2P
  P.s_i32a.resize(nb, s);
  k_flag<<<grid(nb), kT, 0, s>>>(nb, P.x_off.p, nullptr, 1, P.s_i32a.p);
  FMM_LAUNCH_CHECK();
  P.nxboxes = compact(P, nb, P.s_i32a.p, P.xboxes);
  P.xslot.resize(nb, s);
  FMM_CUDA(cudaMemsetAsync(P.xslot.p, 0xff, sizeof(int32_t) * nb, s));
  if (P.nxboxes > 0) {
    k_slot_of<<<grid(P.nxboxes), kT, 0, s>>>(P.nxboxes, P.xboxes.p, P.xslot.p);
    FMM_LAUNCH_CHECK();
  }
  k_flag<<<grid(nb), kT, 0, s>>>(nb, P.w_off.p, P.box_nchild.p, 2, P.s_i32a.p);
  FMM_LAUNCH_CHECK();
  P.nwleaves = compact(P, nb, P.s_i32a.p, P.wleaves);

  build_m2l_tiles(P);
}

}  // namespace fmm

// m2l.cu -- per-level multipole-to-local translation (§2.2: the part of the
// FMM where most of the time goes; translation operators stored as matrices
// and applied as a dense contraction, with one operator per relative offset
// thanks to translational invariance).
//
// One CTA = TILE target boxes of one level with the same octant parity, so
// their interaction-list sources all sit on one 6x6x6 slot grid around the
// parent neighbourhood.  For every occupied slot the CTA stages the slot's
// operator (input-major, k-chunked) and the targets' source multipoles in
// shared memory and accumulates in registers; targets without a source in
// that slot contribute a zero row.  Each target's sum runs over slots in a
// fixed order, so results do not depend on how targets are grouped.
#include "async_copy.cuh"
#include "eval_kernels.cuh"
#include "m2l_config.cuh"

namespace fmm {

namespace {

template <typename T, int TILE, int TPT, int RPT>
__global__ void __launch_bounds__(kM2LThreads)
    k_m2l(int p, const M2LTile *__restrict__ tiles, const int32_t *__restrict__ order,
          const int32_t *__restrict__ voff, const int32_t *__restrict__ vidx,
          const BoxGeo *__restrict__ geo, const T *__restrict__ M, const T *__restrict__ ops,
          T *__restrict__ L) {
  constexpr int TG = TILE / TPT;
  constexpr int RG = kM2LThreads / TG;
  constexpr int NCP = RG * RPT;
  constexpr int KC = kM2LKC;
  constexpr int MP = TILE + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *Ts = reinterpret_cast<T *>(smem_raw);  // [KC][NCP]
  T *Ms = Ts + KC * NCP;                     // [KC][MP]
  int32_t *src = reinterpret_cast<int32_t *>(Ms + KC * MP);  // [216][TILE]
  int32_t *used = src + 216 * TILE;                           // [216]
  int32_t *tgt = used + 216;                                  // [TILE]

  const int nc = ncoef(p), ld = coef_pitch(p);
  const M2LTile tile = tiles[blockIdx.x];
  const int tid = threadIdx.x;
  for (int i = tid; i < 216 * TILE; i += kM2LThreads) src[i] = -1;
  for (int i = tid; i < 216; i += kM2LThreads) used[i] = 0;
  for (int i = tid; i < TILE; i += kM2LThreads) tgt[i] = i < tile.count ? order[tile.start + i] : -1;
  __syncthreads();
  const int px = tile.parity & 1, py = (tile.parity >> 1) & 1, pz = (tile.parity >> 2) & 1;
  for (int t = tid >> 5; t < tile.count; t += kM2LThreads / 32) {
    const int32_t B = tgt[t];
    const BoxGeo gb = geo[B];
    for (int32_t e = voff[B] + (tid & 31); e < voff[B + 1]; e += 32) {
      const int32_t A = vidx[e];
      const BoxGeo ga = geo[A];
      const int sx = ga.ix - gb.ix + 2 + px, sy = ga.iy - gb.iy + 2 + py, sz = ga.iz - gb.iz + 2 + pz;
      if ((unsigned)sx < 6u && (unsigned)sy < 6u && (unsigned)sz < 6u) {  // always, by construction
        const int slot = (sx * 6 + sy) * 6 + sz;
        src[slot * TILE + t] = A;
        used[slot] = 1;
      }
    }
  }
  __syncthreads();

  const int rg = tid % RG, tg = tid / RG;
  T acc[TPT][RPT];
#pragma unroll
  for (int j = 0; j < TPT; ++j)
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[j][i] = T(0);

  for (int slot = 0; slot < 216; ++slot) {
    if (!used[slot]) continue;
    const int sx = slot / 36, sy = (slot / 6) % 6, sz = slot % 6;
    const int dx = 2 + px - sx, dy = 2 + py - sy, dz = 2 + pz - sz;  // target - source anchor
    const T *op = ops + (size_t)((dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)) * nc * nc;
    for (int kc = 0; kc < nc; kc += KC) {
      __syncthreads();
      for (int i = tid; i < KC * NCP; i += kM2LThreads) {
        const int k = i / NCP, r = i - k * NCP;
        Ts[i] = (kc + k < nc && r < nc) ? op[(size_t)(kc + k) * nc + r] : T(0);
      }
      for (int i = tid; i < KC * TILE; i += kM2LThreads) {
        const int t = i / KC, k = i - t * KC;
        const int32_t A = src[slot * TILE + t];
        Ms[k * MP + t] = (A >= 0 && kc + k < nc) ? M[(size_t)A * ld + kc + k] : T(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int k = 0; k < KC; ++k) {
        T mv[TPT], tv[RPT];
#pragma unroll
        for (int j = 0; j < TPT; ++j) mv[j] = Ms[k * MP + tg * TPT + j];
#pragma unroll
        for (int i = 0; i < RPT; ++i) tv[i] = Ts[k * NCP + rg + RG * i];
#pragma unroll
        for (int j = 0; j < TPT; ++j)
#pragma unroll
          for (int i = 0; i < RPT; ++i) acc[j][i] = fma(tv[i], mv[j], acc[j][i]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < TPT; ++j) {
    const int t = tg * TPT + j;
    if (t < tile.count) {
      const int32_t B = tgt[t];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = rg + RG * i;
        if (r < nc) L[(size_t)B * ld + r] = acc[j][i];
      }
    }
  }
}

template <typename T, int TILE, int TPT, int RPT>
void run(int p, int64_t ntiles, const M2LTile *tiles, const int32_t *order, const int32_t *voff,
         const int32_t *vidx, const BoxGeo *geo, const T *M, const T *ops, T *L, cudaStream_t s) {
  constexpr int TG = TILE / TPT, RG = kM2LThreads / TG, NCP = RG * RPT;
  size_t smem = sizeof(T) * (size_t)kM2LKC * (NCP + TILE + 1) + sizeof(int32_t) * (216 * TILE + 216 + TILE);
  auto kern = k_m2l<T, TILE, TPT, RPT>;
  FMM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)ntiles, kM2LThreads, smem, s>>>(p, tiles, order, voff, vidx, geo, M, ops, L);
  FMM_LAUNCH_CHECK();
}

// ------------------------------------------------------ plan-time tables
// One CTA per tile: src[tile][slot][t] = source box of target t in that slot
// (-1 if none) and the ascending list of occupied slots.  The sources of
// target B are its V list, taken straight from its definition: the children
// of the colleagues of parent(B) that are not adjacent to B (same level, so
// adjacency is a Chebyshev distance of at most 1).  The V-list CSR itself is
// not needed on this path.
__global__ void k_m2l_table(int tile_size, const M2LTile *__restrict__ tiles,
                            const int32_t *__restrict__ order, const int32_t *__restrict__ parent,
                            const int32_t *__restrict__ child, const int32_t *__restrict__ nchild,
                            const int32_t *__restrict__ col, const int32_t *__restrict__ ncol,
                            const BoxGeo *__restrict__ geo, int32_t *__restrict__ table,
                            int16_t *__restrict__ slots, int32_t *__restrict__ nslots) {
  __shared__ int32_t used[216];
  const M2LTile tile = tiles[blockIdx.x];
  int32_t *tab = table + (size_t)blockIdx.x * 216 * tile_size;
  for (int i = threadIdx.x; i < 216 * tile_size; i += blockDim.x) tab[i] = -1;
  for (int i = threadIdx.x; i < 216; i += blockDim.x) used[i] = 0;
  __syncthreads();
  const int px = tile.parity & 1, py = (tile.parity >> 1) & 1, pz = (tile.parity >> 2) & 1;
  for (int t = threadIdx.x >> 5; t < tile.count; t += blockDim.x >> 5) {
    const int32_t B = order[tile.start + t];
    const BoxGeo gb = geo[B];
    const int32_t P = parent[B];
    const int nco = ncol[P];
    for (int e = threadIdx.x & 31; e < 8 * nco; e += 32) {
      const int32_t C = col[26 * (int64_t)P + (e >> 3)];
      if ((e & 7) >= nchild[C]) continue;
      const int32_t A = child[C] + (e & 7);
      const BoxGeo ga = geo[A];
      const int dx = ga.ix - gb.ix, dy = ga.iy - gb.iy, dz = ga.iz - gb.iz;
      if (max(abs(dx), max(abs(dy), abs(dz))) <= 1) continue;  // adjacent: near field
      const int sx = dx + 2 + px, sy = dy + 2 + py, sz = dz + 2 + pz;
      if ((unsigned)sx < 6u && (unsigned)sy < 6u && (unsigned)sz < 6u) {  // always, by construction
        const int slot = (sx * 6 + sy) * 6 + sz;
        tab[slot * tile_size + t] = A;
        used[slot] = 1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // compact the occupied slots in order
    int base = 0;
    for (int s0 = 0; s0 < 216; s0 += 32) {
      const int sl = s0 + threadIdx.x;
      const bool u = sl < 216 && used[sl];
      const unsigned mask = __ballot_sync(0xffffffffu, u);
      if (u) slots[(size_t)blockIdx.x * 216 + base + __popc(mask & ((1u << threadIdx.x) - 1u))] = (int16_t)sl;
      base += __popc(mask);
    }
    if (threadIdx.x == 0) nslots[blockIdx.x] = base;
  }
}

// The same table from explicit per-target source rows (CSR): the dual-tree
// pairs that fall into the tile's offset window.
__global__ void k_m2l_table_csr(int tile_size, const M2LTile *__restrict__ tiles,
                                const int32_t *__restrict__ order, const int32_t *__restrict__ off,
                                const int32_t *__restrict__ idx, const BoxGeo *__restrict__ geo,
                                int32_t *__restrict__ table, int16_t *__restrict__ slots,
                                int32_t *__restrict__ nslots) {
  __shared__ int32_t used[216];
  const M2LTile tile = tiles[blockIdx.x];
  int32_t *tab = table + (size_t)blockIdx.x * 216 * tile_size;
  for (int i = threadIdx.x; i < 216 * tile_size; i += blockDim.x) tab[i] = -1;
  for (int i = threadIdx.x; i < 216; i += blockDim.x) used[i] = 0;
  __syncthreads();
  const int px = tile.parity & 1, py = (tile.parity >> 1) & 1, pz = (tile.parity >> 2) & 1;
  for (int t = threadIdx.x >> 5; t < tile.count; t += blockDim.x >> 5) {
    const int32_t B = order[tile.start + t];
    const BoxGeo gb = geo[B];
    for (int32_t e = off[B] + (threadIdx.x & 31); e < off[B + 1]; e += 32) {
      const int32_t A = idx[e];
      const BoxGeo ga = geo[A];
      const int sx = ga.ix - gb.ix + 2 + px, sy = ga.iy - gb.iy + 2 + py, sz = ga.iz - gb.iz + 2 + pz;
      if ((unsigned)sx < 6u && (unsigned)sy < 6u && (unsigned)sz < 6u) {  // always, by construction
        const int slot = (sx * 6 + sy) * 6 + sz;
        tab[slot * tile_size + t] = A;
        used[slot] = 1;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int base = 0;
    for (int s0 = 0; s0 < 216; s0 += 32) {
      const int sl = s0 + threadIdx.x;
      const bool u = sl < 216 && used[sl];
      const unsigned mask = __ballot_sync(0xffffffffu, u);
      if (u) slots[(size_t)blockIdx.x * 216 + base + __popc(mask & ((1u << threadIdx.x) - 1u))] = (int16_t)sl;
      base += __popc(mask);
    }
    if (threadIdx.x == 0) nslots[blockIdx.x] = base;
  }
}

// ------------------------------------------------------------ rotated M2L
// Per tile (targets of one level and octant parity) and occupied slot: the
// sources' multipoles are staged, rotated so that the slot's offset lies on
// the z axis (block-diagonal by degree), translated along z (only equal
// orders couple), rotated back and added to the targets' locals.  The
// targets go through in groups of TT so that three TT x (p+1)^2 buffers fit
// in shared memory; every thread keeps up to kRotItems local coefficients of
// the group in registers across the slots.  2(p+1)(2p+1)(2p+3)/3 + ~(p+1)^3/3
// multiply-adds per pair against (p+1)^4 for the dense operator.
constexpr int kRotThreads = 256;
constexpr int kRotItems = 16;

__device__ __forceinline__ int rot_degree(int k) {
  int n = (int)sqrtf((float)k);
  while (n * n > k) --n;
  while ((n + 1) * (n + 1) <= k) ++n;
  return n;
}

template <typename T>
__global__ void __launch_bounds__(kRotThreads)
    k_m2l_rot(int p, int TT, int tile_size, const M2LTile *__restrict__ tiles,
              const int32_t *__restrict__ table, const int16_t *__restrict__ slots,
              const int32_t *__restrict__ nslots, const int32_t *__restrict__ order,
              const T *__restrict__ M, const T *__restrict__ rot, const T *__restrict__ zt,
              T *__restrict__ L) {
  extern __shared__ __align__(16) unsigned char rot_smem[];
  const int nc = (p + 1) * (p + 1), ld = coef_pitch(p), P1 = p + 1;
  const size_t nrot = (size_t)(p + 1) * (2 * p + 1) * (2 * p + 3) / 3;
  T *Ms = reinterpret_cast<T *>(rot_smem), *Mb = Ms + TT * nc, *Lb = Mb + TT * nc;
  const M2LTile tile = tiles[blockIdx.x];
  const int px = tile.parity & 1, py = (tile.parity >> 1) & 1, pz = (tile.parity >> 2) & 1;
  const int32_t *tab = table + (size_t)blockIdx.x * 216 * tile_size;
  const int16_t *sl = slots + (size_t)blockIdx.x * 216;
  const int ns = nslots[blockIdx.x];
  const int tid = threadIdx.x, items = TT * nc;
  for (int t0 = 0; t0 < tile.count; t0 += TT) {
    const int tc = min(TT, tile.count - t0);
    T acc[kRotItems];
#pragma unroll
    for (int q = 0; q < kRotItems; ++q) acc[q] = T(0);
    for (int j = 0; j < ns; ++j) {
      const int slot = sl[j];
      const int sx = slot / 36, sy = (slot / 6) % 6, sz = slot % 6;
      const int code = (2 + px - sx + 3) * 49 + (2 + py - sy + 3) * 7 + (2 + pz - sz + 3);
      const T *Dm = rot + (size_t)code * 2 * nrot, *Dl = Dm + nrot;
      const T *z = zt + (size_t)code * P1 * P1;
      __syncthreads();  // the previous slot's buffers are consumed
      for (int i = tid; i < items; i += kRotThreads) {
        const int t = i / nc, k = i - t * nc;
        const int32_t S = t < tc ? tab[(size_t)slot * tile_size + t0 + t] : -1;
        Ms[i] = S >= 0 ? M[(int64_t)S * ld + k] : T(0);
      }
      __syncthreads();
      for (int i = tid; i < items; i += kRotThreads) {  // M' = A M, degree by degree
        const int t = i / nc, k = i - t * nc, n = rot_degree(k), w = 2 * n + 1;
        const T *row = Dm + (size_t)n * (2 * n - 1) * (2 * n + 1) / 3 + (size_t)(k - n * n) * w;
        const T *x = Ms + t * nc + n * n;
        T s = T(0);
        for (int c = 0; c < w; ++c) s += row[c] * x[c];
        Mb[i] = s;
      }
      __syncthreads();
      for (int i = tid; i < items; i += kRotThreads) {  // translation along z
        const int t = i / nc, k = i - t * nc, n = rot_degree(k), mm = k - n * n - n;
        const int am = mm < 0 ? -mm : mm;
        const T *zr = z + n * P1;
        const T *x = Mb + t * nc;
        T s = T(0);
        for (int kk = am; kk <= p; ++kk) s += zr[kk] * x[kk * kk + kk + mm];
        Lb[i] = ((n + am) & 1) ? -s : s;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kRotItems; ++q) {  // L += B L', into the owned coefficients
        const int i = tid + q * kRotThreads;
        if (i < items) {
          const int t = i / nc, k = i - t * nc, n = rot_degree(k), w = 2 * n + 1;
          const T *row = Dl + (size_t)n * (2 * n - 1) * (2 * n + 1) / 3 + (size_t)(k - n * n) * w;
          const T *x = Lb + t * nc + n * n;
          T s = T(0);
          for (int c = 0; c < w; ++c) s += row[c] * x[c];
          acc[q] += s;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kRotItems; ++q) {
      const int i = tid + q * kRotThreads;
      if (i < items) {
        const int t = i / nc, k = i - t * nc;
        if (t < tc) L[(int64_t)order[tile.start + t0 + t] * ld + k] = acc[q];
      }
    }
  }
}

// ------------------------------------------------- staged FP32 M2L kernel

constexpr int kStagedTile = 64, kStagedTPT = 4, kStagedRG = 16;

// Per occupied slot: the slot's padded operator rows [NCP][ld] and the 64
// targets' source multipoles [64][ld] are copied into one of two shared
// stages with cp.async while the other stage is contracted; each thread owns
// 4 targets x RPT rows and reads both operands as float4 along k.
template <int RPT>
__global__ void __launch_bounds__(kM2LThreads)
    k_m2l_staged(int p, const M2LTile *__restrict__ tiles, const int32_t *__restrict__ table,
                 const int16_t *__restrict__ slots, const int32_t *__restrict__ nslots,
                 const int32_t *__restrict__ order, const float *__restrict__ M,
                 const float *__restrict__ opsp, float *__restrict__ L) {
  constexpr int NCP = kStagedRG * RPT;
  constexpr int TILE = kStagedTile, TPT = kStagedTPT;
  extern __shared__ float4 smem4[];
  float *sm = reinterpret_cast<float *>(smem4);
  const int nc = ncoef(p), ld = coef_pitch(p), cpr = ld / 4;
  const int stage = (NCP + TILE) * ld;
  const int tid = threadIdx.x, rg = tid % kStagedRG, tg = tid / kStagedRG;
  const M2LTile tile = tiles[blockIdx.x];
  const int ns = nslots[blockIdx.x];
  const int px = tile.parity & 1, py = (tile.parity >> 1) & 1, pz = (tile.parity >> 2) & 1;
  const int32_t *tab = table + (size_t)blockIdx.x * 216 * TILE;
  const int16_t *sl = slots + (size_t)blockIdx.x * 216;

  auto issue = [&](int j, int buf) {
    const int slot = sl[j];
    const int sx = slot / 36, sy = (slot / 6) % 6, sz = slot % 6;
    const int code = (2 + px - sx + 3) * 49 + (2 + py - sy + 3) * 7 + (2 + pz - sz + 3);
    const float *op = opsp + (size_t)code * NCP * ld;
    float *Ts = sm + buf * stage;
    float *Ms = Ts + NCP * ld;
    for (int c = tid; c < NCP * cpr; c += kM2LThreads) cp_async16(Ts + 4 * c, op + 4 * c, 16);
    for (int c = tid; c < TILE * cpr; c += kM2LThreads) {
      const int t = c / cpr, kk = c - t * cpr;
      const int32_t A = tab[slot * TILE + t];
      cp_async16(Ms + t * ld + 4 * kk, A >= 0 ? M + (size_t)A * ld + 4 * kk : M, A >= 0 ? 16 : 0);
    }
    cp_async_commit();
  };

  float acc[TPT][RPT];
#pragma unroll
  for (int j = 0; j < TPT; ++j)
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[j][i] = 0.f;

  if (ns > 0) issue(0, 0);
  for (int j = 0; j < ns; ++j) {
    if (j + 1 < ns) {
      issue(j + 1, (j + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float *Ts = sm + (j & 1) * stage;
    const float *Ms = Ts + NCP * ld;
#pragma unroll 3
    for (int k4 = 0; k4 < cpr; ++k4) {
      float4 mv[TPT], tv[RPT];
#pragma unroll
      for (int q = 0; q < TPT; ++q)
        mv[q] = *reinterpret_cast<const float4 *>(Ms + (tg * TPT + q) * ld + 4 * k4);
#pragma unroll
      for (int i = 0; i < RPT; ++i)
        tv[i] = *reinterpret_cast<const float4 *>(Ts + (rg + kStagedRG * i) * ld + 4 * k4);
#pragma unroll
      for (int q = 0; q < TPT; ++q)
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          float a = acc[q][i];
          a = fmaf(tv[i].x, mv[q].x, a);
          a = fmaf(tv[i].y, mv[q].y, a);
          a = fmaf(tv[i].z, mv[q].z, a);
          a = fmaf(tv[i].w, mv[q].w, a);
          acc[q][i] = a;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int t = tg * TPT + q;
    if (t < tile.count) {
      const int32_t B = order[tile.start + t];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = rg + kStagedRG * i;
        if (r < nc) L[(size_t)B * ld + r] = acc[q][i];
      }
    }
  }
}

template <int RPT>
void run_staged(int p, int64_t ntiles, const M2LTile *tiles, const int32_t *table,
                const int16_t *slots, const int32_t *nslots, const int32_t *order, const float *M,
                const float *opsp, float *L, cudaStream_t s) {
  constexpr int NCP = kStagedRG * RPT;
  const size_t smem = 2 * sizeof(float) * (size_t)(NCP + kStagedTile) * coef_pitch(p);
  auto kern = k_m2l_staged<RPT>;
  FMM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)ntiles, kM2LThreads, smem, s>>>(p, tiles, table, slots, nslots, order, M, opsp, L);
  FMM_LAUNCH_CHECK();
}

}  // namespace

template <typename T>
void launch_m2l(int p, int64_t ntiles, const M2LTile *tiles, int tile, const int32_t *order,
                const int32_t *voff, const int32_t *vidx, const BoxGeo *geo, const T *M,
                const T *ops, T *L, cudaStream_t s) {
  if (ntiles == 0) return;
  const M2LShape sh = m2l_shape(p);
  if (sh.tile != tile) throw Error(FMM_ERR_INVALID_ARG, "M2L tile size does not match the plan");
#define FMM_M2L_CASE(TL, TP, RP) \
  if (sh.tile == TL && sh.tpt == TP && sh.rpt == RP) return run<T, TL, TP, RP>(p, ntiles, tiles, order, voff, vidx, geo, M, ops, L, s);
  FMM_M2L_CASE(64, 4, 1)
  FMM_M2L_CASE(64, 4, 2)
  FMM_M2L_CASE(64, 4, 3)
  FMM_M2L_CASE(64, 4, 4)
  FMM_M2L_CASE(64, 4, 6)
  FMM_M2L_CASE(64, 4, 7)
  FMM_M2L_CASE(64, 4, 8)
  FMM_M2L_CASE(32, 2, 16)
  FMM_M2L_CASE(16, 1, 28)
#undef FMM_M2L_CASE
  throw Error(FMM_ERR_UNSUPPORTED, "no M2L tile shape for this order");
}

void launch_m2l_staged(int p, int64_t ntiles, const M2LTile *tiles, const int32_t *table,
                       const int16_t *slots, const int32_t *nslots, const int32_t *order,
                       const float *M, const float *opsp, float *L, cudaStream_t s) {
  if (ntiles == 0) return;
  switch (m2l_rows(p) / kStagedRG) {
    case 1: return run_staged<1>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 2: return run_staged<2>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 3: return run_staged<3>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 4: return run_staged<4>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 5: return run_staged<5>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 6: return run_staged<6>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 7: return run_staged<7>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
    case 8: return run_staged<8>(p, ntiles, tiles, table, slots, nslots, order, M, opsp, L, s);
  }
  throw Error(FMM_ERR_UNSUPPORTED, "staged M2L supports orders up to 10");
}

void build_m2l_tables(fmm_plan_impl &P) {
  cudaStream_t s = P.stream;
  const int64_t nt = P.nm2l_tiles;
  if (nt == 0) return;
  P.m2l_src.resize((size_t)nt * 216 * P.m2l_tile_size, s);
  P.m2l_slots.resize((size_t)nt * 216, s);
  P.m2l_nslots.resize((size_t)nt, s);
  if (P.dual)
    k_m2l_table_csr<<<(unsigned)nt, 256, 0, s>>>(P.m2l_tile_size, P.m2l_tiles.p, P.m2l_order.p,
                                                 P.dt_toff.p, P.dt_tidx.p, P.box_geo.p, P.m2l_src.p,
                                                 P.m2l_slots.p, P.m2l_nslots.p);
  else
    k_m2l_table<<<(unsigned)nt, 256, 0, s>>>(P.m2l_tile_size, P.m2l_tiles.p, P.m2l_order.p,
                                              P.box_parent.p, P.box_child.p, P.box_nchild.p,
                                              P.colleagues.p, P.ncolleagues.p, P.box_geo.p,
                                              P.m2l_src.p, P.m2l_slots.p, P.m2l_nslots.p);
  FMM_LAUNCH_CHECK();
}

template <typename T>
void launch_m2l_rot(int p, int64_t ntiles, const M2LTile *tiles, int tile_size, const int32_t *table,
                    const int16_t *slots, const int32_t *nslots, const int32_t *order, const T *M,
                    const T *rot, const T *zt, T *L, cudaStream_t s) {
  if (ntiles == 0) return;
  const int nc = ncoef(p);
  const int TT = std::min(32, kRotThreads * kRotItems / nc);
  const size_t smem = sizeof(T) * 3 * (size_t)TT * nc;
  if (smem > 48 * 1024)
    FMM_CUDA(cudaFuncSetAttribute(k_m2l_rot<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_m2l_rot<T><<<(unsigned)ntiles, kRotThreads, smem, s>>>(p, TT, tile_size, tiles, table, slots,
                                                            nslots, order, M, rot, zt, L);
  FMM_LAUNCH_CHECK();
}

template void launch_m2l_rot<double>(int, int64_t, const M2LTile *, int, const int32_t *,
                                     const int16_t *, const int32_t *, const int32_t *,
                                     const double *, const double *, const double *, double *,
                                     cudaStream_t);
template void launch_m2l_rot<float>(int, int64_t, const M2LTile *, int, const int32_t *,
                                    const int16_t *, const int32_t *, const int32_t *, const float *,
                                    const float *, const float *, float *, cudaStream_t);

template void launch_m2l<float>(int, int64_t, const M2LTile *, int, const int32_t *, const int32_t *,
                                const int32_t *, const BoxGeo *, const float *, const float *, float *,
                                cudaStream_t);
template void launch_m2l<double>(int, int64_t, const M2LTile *, int, const int32_t *, const int32_t *,
                                 const int32_t *, const BoxGeo *, const double *, const double *,
                                 double *, cudaStream_t);

}  // namespace fmm

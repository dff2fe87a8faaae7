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

  const int nc = ncoef(p);
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
        Ms[k * MP + t] = (A >= 0 && kc + k < nc) ? M[(size_t)A * nc + kc + k] : T(0);
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
        if (r < nc) L[(size_t)B * nc + r] = acc[j][i];
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

template void launch_m2l<float>(int, int64_t, const M2LTile *, int, const int32_t *, const int32_t *,
                                const int32_t *, const BoxGeo *, const float *, const float *, float *,
                                cudaStream_t);
template void launch_m2l<double>(int, int64_t, const M2LTile *, int, const int32_t *, const int32_t *,
                                 const int32_t *, const BoxGeo *, const double *, const double *,
                                 double *, cudaStream_t);

}  // namespace fmm

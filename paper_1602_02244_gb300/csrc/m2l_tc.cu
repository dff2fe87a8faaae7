// m2l_tc.cu -- per-level M2L on the 5th-generation tensor cores (§2.2: the
// translation that dominates FMM run time, applied as a dense contraction
// with one precomputed operator per relative offset).
//
// A CTA owns 128 target boxes of one level with the same octant parity (the
// M = 128 rows of the MMA).  For every occupied offset slot it contracts
//   D[t][n] += sum_k M_src(t)[k] T_slot[n][k]     (N = rows of the operator)
// with tcgen05.mma kind::tf32.  FP32 accuracy comes from the three-product
// split
//   A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi,
// where X_hi is X rounded to TF32 and X_lo is X - X_hi rounded to TF32.  The
// hi and lo operator halves are stored one after the other, so they form a
// single 2N-row operand: per K step one MMA computes [A_hi B_hi | A_hi B_lo]
// into 2N accumulator columns and a second adds A_lo B_hi to the first N.
// The multipoles are split once per evaluation (k_split_tf32) and the
// operators at plan time, already in the layouts the MMA reads.  Each slot is
// contracted in K chunks of 32; chunks are copied into a ring of
// shared-memory stages while the tensor core works on earlier stages, and a
// stage is refilled only after the mbarrier signalled by tcgen05.commit says
// its MMAs have finished.  All waits are bounded; a timeout sets an error
// word and the CTA still frees its tensor memory.
//
// The FP16 form (kind::f16) carries the same 22 significant bits in half the
// bytes and at twice the MMA rate: X = X_hi + X_lo with both halves FP16.
// FP16's exponent range is made to fit by exact power-of-two scalings: the
// operators are balanced once per order, T'[n][k] = T[n][k] 2^-(e_n + f_k)
// (all |T'| <= 1); each source multipole is stored as
// M'_k = M_k 2^(f_k) / s_A with s_A the power of two at or above its largest
// |M_k 2^(f_k)|; the drain warps add each finished slot as s_A x (slot sum),
// and the stored local is 2^(e_n) x the accumulated sum.  Rounding stays
// relative to the largest entry of each row, as in FP32.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include <type_traits>

#include <cuda_fp16.h>

#include "async_copy.cuh"
#include "eval_kernels.cuh"
#include "m2l_config.cuh"
#include "tcgen05.cuh"

namespace fmm {

namespace {

constexpr int kTcTile = 128;     // targets per CTA = MMA M
constexpr int kTcKC = 32;        // K per stage (TF32); a stage row is 128 bytes in both forms
constexpr int kTcRowBytes = 128;
constexpr long long kTcWaitCycles = 400000000ll;  // ~0.2 s: far beyond any legitimate wait

// Mhi/Mlo[b][k] (pitch kt, zero beyond the nc coefficients) from M[b][k] (pitch ld)
__global__ void k_split_tf32(int64_t nb, int nc, int ld, int kt, const float *__restrict__ M,
                             float *__restrict__ Mhi, float *__restrict__ Mlo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * kt) return;
  const int64_t b = i / kt;
  const int k = (int)(i - b * kt);
  float hi = 0.f, lo = 0.f;
  if (k < nc) tc::split_tf32(M[b * ld + k], hi, lo);
  Mhi[i] = hi;
  Mlo[i] = lo;
}

__host__ __device__ constexpr int tc_k(int p) { return (ncoef(p) + kTcKC - 1) / kTcKC * kTcKC; }

// FP16 form: M'_b = M_b[k] colscale[k] / s_b split into FP16 halves (pitch kt
// halves, zero beyond nc), s_b = the power of two at or above max |M_b[k]
// colscale[k]| (1 for an all-zero row); a warp per box
__global__ void k_split_f16(int64_t nb, int nc, int ld, int kt, const float *__restrict__ M,
                            const float *__restrict__ colscale, __half *__restrict__ Mhi,
                            __half *__restrict__ Mlo, float *__restrict__ mscale) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nb) return;
  float mx = 0.f;
  for (int k = lane; k < nc; k += 32) mx = fmaxf(mx, fabsf(M[b * ld + k] * colscale[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // power of two >= mx: 2^ceil(log2 mx) from the exponent bits (exact)
  int e = 0;
  if (mx > 0.f) {
    const float m = frexpf(mx, &e);  // mx = m 2^e, 0.5 <= m < 1
    if (m == 0.5f) e -= 1;           // mx is itself a power of two
  }
  const float sc = mx > 0.f ? ldexpf(1.f, e) : 1.f, inv = mx > 0.f ? ldexpf(1.f, -e) : 1.f;
  if (lane == 0) mscale[b] = sc;
  for (int k = lane; k < kt; k += 32) {
    const float v = k < nc ? M[b * ld + k] * colscale[k] * inv : 0.f;
    const __half h = __float2half_rn(v);
    Mhi[b * kt + k] = h;
    Mlo[b * kt + k] = __float2half_rn(v - __half2float(h));
  }
}

// The tensor core's FP32 accumulation does not round to nearest, so its error
// grows with the number of accumulations into one tile.  Every slot therefore
// starts a fresh accumulator (two in tensor memory, by slot parity), and the
// finished slot is drained with tcgen05.ld into per-thread FP32 registers
// (round-to-nearest adds) while the tensor core works on the next slot.
//
// Warp roles (no block-wide barrier between setup and teardown):
//   warps 0-3  drain: warp w owns tensor-memory lanes 32w..32w+31, i.e. the
//              targets 32w..32w+31 of the tile, and adds finished slots into
//              registers; they write L at the end;
//   warp 4     one thread issues the MMAs and the tcgen05.commit arrivals;
//   warps 5-8  producers: gather the A rows (source multipoles) of each
//              (slot, K chunk) stage with cp.async, fence their writes into
//              the async proxy and arrive on the stage's `full` barrier; one
//              of them also moves the stage's operator slab with a bulk async
//              copy that completes its bytes on the same barrier.
// Barriers: full[s] (128 producer arrivals once the rows have landed, plus
// one arrival that announces the slab's bytes, which the bulk copy completes)
// -> MMA; empty[s] (commit) -> producers; accf[a] (commit after a slot) ->
// drain; acce[a] (128 drain arrivals) -> MMA before it overwrites
// accumulator a.  The MMA thread thus waits on one barrier per stage: each
// of its waits costs a few hundred cycles in which the tensor core idles.
constexpr int kTcDrainWarps = 4;
constexpr int kTcProdWarps = 4;
constexpr int kTcProdThreads = 32 * kTcProdWarps;
constexpr int kTcThreads = 32 * (kTcDrainWarps + 1 + kTcProdWarps);
constexpr int kTcRowsPerProd = kTcTile * (kTcKC / 4) / kTcProdThreads;  // 8

// Wait for a phase of an mbarrier; gives up after kTcWaitCycles or as soon as
// another thread of the CTA gave up (the abort word), so that one timeout does
// not make every later wait of the CTA run to its own limit.  A phase that has
// already completed returns before the clock is read: in the thread that
// issues the MMAs, the clock read and the abort-word load cost ~170 cycles
// per wait (measured), time in which no MMA is issued.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t parity, volatile int *abort) {
  if (tc::mbar_try_wait(mbar, parity)) return true;
  const long long t0 = clock64();
  while (!tc::mbar_try_wait(mbar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > kTcWaitCycles) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

// F16: the FP16 form (operands of 2 bytes, kind::f16, scalings as described
// at the top of the file); else the TF32 form.  Either way a stage row holds
// 128 bytes of K (32 TF32 or 64 FP16 values), and the last K chunk of an
// FP16 slot may hold only 32 values (64 bytes, two MMA K steps).
template <int NT, int NSTAGE, bool F16>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_m2l_tc(int p, int kt, const M2LTile *__restrict__ tiles,
             const int32_t *__restrict__ table,
             const int16_t *__restrict__ slots, const int32_t *__restrict__ nslots,
             const int32_t *__restrict__ order, const unsigned char *__restrict__ Mhi,
             const unsigned char *__restrict__ Mlo, const unsigned char *__restrict__ opt,
             const float *__restrict__ mscale, const float *__restrict__ rowscale,
             float *__restrict__ L, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ uint64_t full[NSTAGE], empty[NSTAGE], accf[2], acce[2], done;
  __shared__ uint32_t tslot;
  __shared__ int abort_word;
  __shared__ int16_t s_slots[216];  // the tile's occupied slots, in order
  volatile int *abort = &abort_word;
  constexpr int N = NT;
  // an accumulator holds [A_hi B_hi + A_lo B_hi | A_hi B_lo]: 2N columns
  constexpr uint32_t kCols = 2 * N <= 32 ? 32 : 2 * N <= 64 ? 64 : 2 * N <= 128 ? 128 : 256;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kEsz = F16 ? 2 : 4;  // operand bytes
  const int nc = ncoef(p), ld = coef_pitch(p);
  const int kt_bytes = kt * kEsz, nch = (kt_bytes + kTcRowBytes - 1) / kTcRowBytes;
  // bytes of K in chunk c (128 except possibly the last FP16 chunk)
  auto chunk_bytes = [&](int c) { return min(kTcRowBytes, kt_bytes - c * kTcRowBytes); };
  constexpr uint32_t a_bytes = kTcTile * kTcRowBytes, b_bytes = (uint32_t)N * kTcRowBytes;
  constexpr uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;  // a multiple of 1024
  // the swizzled A tiles need a 1024-byte-aligned base (1 KB of slack is allocated)
  unsigned char *sm = sm_raw + ((1024u - (tc::smem_addr(sm_raw) & 1023u)) & 1023u);
  const M2LTile tile = tiles[blockIdx.x];
  const int ns = nslots[blockIdx.x];
  const int total = ns * nch;

  if (total == 0) {  // no interaction-list source anywhere in the tile
    for (int i = tid; i < tile.count * nc; i += kTcThreads) {
      const int tt = i / nc, r = i - tt * nc;
      L[(size_t)order[tile.start + tt] * ld + r] = 0.f;
    }
    return;
  }
  if (tid == 0) {
    for (int q = 0; q < NSTAGE; ++q) {
      tc::mbar_init(&full[q], kTcProdThreads + 1);
      tc::mbar_init(&empty[q], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], 32 * kTcDrainWarps);
    }
    tc::mbar_init(&done, 1);
    abort_word = 0;
  }
  for (int j = tid; j < ns; j += kTcThreads) s_slots[j] = slots[(size_t)blockIdx.x * 216 + j];
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;

  float acc[N];
#pragma unroll
  for (int i = 0; i < N; ++i) acc[i] = 0.f;

  if (warp < kTcDrainWarps) {
    // ---------------------------------------------------------------- drain
    // FP16 form: the scale s_A of this row's source in slot j (0 where the
    // slot has no source for this target).  Its two dependent loads (source
    // box, then scale) are pipelined over the slots: at slot j the box of
    // slot j + 2 and the scale of slot j + 1 are requested, so no load is
    // waited for within the slot it was issued in.
    const int t = warp * 32 + lane;
    const int32_t *tab_t = table + (size_t)blockIdx.x * 216 * kTcTile + t;
    auto src_of = [&](int j) { return F16 && j < ns ? tab_t[(int)s_slots[j] * kTcTile] : -1; };
    auto scale_of = [&](int32_t src) { return src >= 0 ? mscale[src] : 0.f; };
    int32_t src_next = src_of(1);
    float sc_next = F16 ? scale_of(src_of(0)) : 1.f;
    for (int j = 0; j < ns; ++j) {
      const int a = j & 1;
      const float sc = sc_next;
      if (F16) {
        const int32_t src_after = src_of(j + 2);
        sc_next = scale_of(src_next);
        src_next = src_after;
      }
      // warp-uniform outcome: tcgen05.ld is a warp-collective instruction
      const bool ok = __all_sync(0xffffffffu, tc_wait(&accf[a], (uint32_t)(j >> 1) & 1, abort));
      if (!ok) break;
      tc::fence_after_sync();
      const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * kCols);
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16], w[16];
        tc::tmem_ld16(base + (uint32_t)c0, v);
        tc::tmem_ld16(base + (uint32_t)(N + c0), w);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (F16) acc[c0 + i] = fmaf(sc, v[i] + w[i], acc[c0 + i]);
          else acc[c0 + i] += v[i] + w[i];
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&acce[a]);
    }
  } else if (warp == kTcDrainWarps) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      // the hi and lo operator slabs are contiguous, i.e. one 2N-row operand
      const uint32_t idesc2 = F16 ? tc::idesc_f16(kTcTile, 2 * N) : tc::idesc_tf32(kTcTile, 2 * N);
      const uint32_t idesc1 = F16 ? tc::idesc_f16(kTcTile, N) : tc::idesc_tf32(kTcTile, N);
      bool ok = true;
      for (int j = 0; j < ns && ok; ++j) {
        const int a = j & 1;
        if (j >= 2) {
          ok = tc_wait(&acce[a], (uint32_t)((j >> 1) - 1) & 1, abort);
          if (!ok) break;
          tc::fence_after_sync();
        }
        const uint32_t dtm = tmem + (uint32_t)(a * kCols);
        for (int c = 0; c < nch; ++c) {
          const int st = j * nch + c;
          ok = tc_wait(&full[st % NSTAGE], (uint32_t)(st / NSTAGE) & 1, abort);
          if (!ok) break;
          tc::fence_after_sync();
          const uint32_t base = tc::smem_addr(sm + (st % NSTAGE) * stage_bytes);
          const uint32_t ah = base, al = base + a_bytes, bh = base + 2 * a_bytes;
          // the operator slab of this chunk: N rows of cb bytes, core-matrix order
          const int cb = chunk_bytes(c);
          const uint32_t sbo = (uint32_t)(cb / 16) * 128;
          for (int ks = 0; ks < cb / 32; ++ks) {
            const uint64_t dah = tc::smem_desc_sw128(ah + (uint32_t)ks * 32);
            const uint64_t dal = tc::smem_desc_sw128(al + (uint32_t)ks * 32);
            const uint64_t dbh = tc::smem_desc(bh + (uint32_t)ks * 256, 128, sbo);
            // A_hi [B_hi; B_lo] into all 2N columns, then A_lo B_hi into the first N
            if (F16) {
              tc::mma_f16(dtm, dah, dbh, idesc2, (c > 0 || ks > 0) ? 1u : 0u);
              tc::mma_f16(dtm, dal, dbh, idesc1, 1u);
            } else {
              tc::mma_tf32(dtm, dah, dbh, idesc2, (c > 0 || ks > 0) ? 1u : 0u);
              tc::mma_tf32(dtm, dal, dbh, idesc1, 1u);
            }
          }
          tc::mma_commit(&empty[st % NSTAGE]);
        }
        if (ok) tc::mma_commit(&accf[a]);
      }
      // every MMA issued above has completed before tensor memory is freed
      tc::mma_commit(&done);
      tc::mbar_wait_bounded(&done, 0, kTcWaitCycles);
    }
  } else {
    // ---------------------------------------------------------------- producers
    // Thread pt copies 16-byte chunk kk of rows rq + 16 i, i < 8, in both
    // halves: the 8 lanes of a row read one 128-byte line of the source and
    // fill the row's 128 swizzled bytes (no bank conflicts).
    // The full barrier of a stage is signalled kLag stages after its copies
    // were issued, so the producer never waits on the MMAs of a stage it has
    // only just handed over.
    constexpr int kLag = NSTAGE - 2;
    const int pt = tid - 32 * (kTcDrainWarps + 1);
    const int kk = pt & 7, rq = pt >> 3;
    const int px = tile.parity & 1, py = (tile.parity >> 1) & 1, pz = (tile.parity >> 2) & 1;
    const int32_t *tab = table + (size_t)blockIdx.x * 216 * kTcTile;
    const size_t lo_off = (size_t)(Mlo - Mhi);
    // missing sources (row -1) are zero-filled by the copy itself (source
    // size 0): pointing them at a shared zero row would make every SM hit the
    // same L2 lines
    const unsigned char *rp[kTcRowsPerProd];
    int rsz[kTcRowsPerProd];
    int32_t next[kTcRowsPerProd];
    int code = 0, next_code = 0;
    auto fetch = [&](int j) {  // source rows and operator code of slot j
      const int slot = s_slots[j];
      const int sx = slot / 36, sy = (slot / 6) % 6, sz = slot % 6;
      next_code = (2 + px - sx + 3) * 49 + (2 + py - sy + 3) * 7 + (2 + pz - sz + 3);
#pragma unroll
      for (int i = 0; i < kTcRowsPerProd; ++i)
        next[i] = tab[slot * kTcTile + rq + 16 * i];
    };
    fetch(0);
    int st = 0, signalled = 0;
    for (; st < total; ++st) {
      const int j = st / nch, c = st - j * nch, s = st % NSTAGE;
      if (st >= NSTAGE && !tc_wait(&empty[s], (uint32_t)(st / NSTAGE - 1) & 1, abort)) break;
      if (c == 0) {
#pragma unroll
        for (int i = 0; i < kTcRowsPerProd; ++i) {
          rp[i] = Mhi + (size_t)(next[i] >= 0 ? next[i] : 0) * kt_bytes + 16 * kk;
          rsz[i] = next[i] >= 0 ? 16 : 0;
        }
        code = next_code;
        if (j + 1 < ns) fetch(j + 1);  // consumed one slot later
      }
      // rows rq + 16 i share (row & 7) = rq & 7, hence the chunk position
      unsigned char *base = sm + s * stage_bytes + tc::sw128_offset(rq, 4 * kk);
      const int cb = chunk_bytes(c);
      if (16 * kk < cb) {  // the MMAs of a 64-byte chunk read its first four 16-byte pieces
#pragma unroll
        for (int i = 0; i < kTcRowsPerProd; ++i) {
          const unsigned char *src = rp[i] + c * kTcRowBytes;
          cp_async16(base + i * 16 * 128, src, rsz[i]);
          cp_async16(base + a_bytes + i * 16 * 128, src + lo_off, rsz[i]);
        }
      }
      if (pt == 0) {  // the operator slab (hi and lo halves) is contiguous: one bulk copy
        const uint32_t slab = 2u * (uint32_t)N * (uint32_t)cb;
        const unsigned char *bsrc = opt + (size_t)code * 2 * N * kt_bytes + (size_t)c * 2 * N * kTcRowBytes;
        tc::mbar_arrive_expect_tx(&full[s], slab);
        tc::bulk_g2s(sm + s * stage_bytes + 2 * a_bytes, bsrc, slab, &full[s]);
      }
      cp_async_commit();
      if (st >= kLag) {  // the stage issued kLag steps ago has landed
        cp_async_wait<kLag>();
        tc::fence_async_shared();
        tc::mbar_arrive(&full[(st - kLag) % NSTAGE]);
        ++signalled;
      }
    }
    cp_async_wait<0>();
    tc::fence_async_shared();
    for (; signalled < st; ++signalled) tc::mbar_arrive(&full[signalled % NSTAGE]);
    if (*abort && pt == 0) {
      // slabs of the last NSTAGE issued stages may still be in flight: their
      // bytes complete those stages' full phases, so waiting (bounded) on
      // them lets the copies land before the CTA's shared memory is released
      for (int q = st - NSTAGE > 0 ? st - NSTAGE : 0; q < st; ++q)
        tc::mbar_wait_bounded(&full[q % NSTAGE], (uint32_t)(q / NSTAGE) & 1, kTcWaitCycles);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  const bool failed = *abort != 0;
  if (failed && tid == 0) atomicExch(err, 1);
  if (!failed && warp < kTcDrainWarps) {
    const int t = warp * 32 + lane;
    if (t < tile.count) {
      const int32_t B = order[tile.start + t];
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (i < nc) L[(size_t)B * ld + i] = F16 ? acc[i] * rowscale[i] : acc[i];
    }
  }
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kCols);
}

// round to the nearest TF32 value, ties away from zero (as cvt.rna.tf32.f32)
float round_tf32_host(float v) {
  uint32_t bits;
  std::memcpy(&bits, &v, 4);
  bits = (bits + 0x1000u) & 0xFFFFE000u;
  float h;
  std::memcpy(&h, &bits, 4);
  return h;
}

}  // namespace

// operand sizes: N = m2l_rows(p) output rows (a multiple of 16, the MMA N and
// tensor-memory columns), K = tc_k(p) input coefficients (a multiple of the
// 32-wide K stage)
size_t m2l_tc_operator_floats(int p) {
  return (size_t)343 * (tc_k(p) / kTcKC) * 2 * m2l_rows(p) * kTcKC;
}

size_t m2l_tc_pitch(int p) { return (size_t)tc_k(p); }

// operators for the tensor-core path: per offset code and K chunk, the hi and
// lo halves of T[n][k] (n, k < nc; zero padded to N rows and K columns) in
// the K-major core-matrix layout of an N x 32 operand
void pack_m2l_tc_operators(int p, const double *m2l_in_major, float *out) {
  const int nc = ncoef(p), N = m2l_rows(p), nch = tc_k(p) / kTcKC;
  const size_t nn = (size_t)nc * nc, slab = (size_t)N * kTcKC;
  for (int code = 0; code < 343; ++code)
    for (int c = 0; c < nch; ++c) {
      float *hi = out + ((size_t)code * nch + c) * 2 * slab, *lo = hi + slab;
      for (int n = 0; n < N; ++n)
        for (int kl = 0; kl < kTcKC; ++kl) {
          const int k = c * kTcKC + kl;
          const float v = (n < nc && k < nc) ? (float)m2l_in_major[code * nn + (size_t)k * nc + n] : 0.f;
          const float h = round_tf32_host(v);
          const uint32_t o = tc::kmajor_offset(n, kl, kTcKC) / 4;
          hi[o] = h;
          lo[o] = round_tf32_host(v - h);
        }
    }
}

// FP16 form of the operators: exact power-of-two balancing of the 343
// scale-free matrices, T'[n][k] = T[n][k] 2^-(e_n + f_k) with every |T'| <= 1
// (alternating row and column maxima over all offsets, a few rounds), then
// per offset code and K chunk the hi and lo FP16 halves of T' in the K-major
// core-matrix layout of an N x kc operand (kc = 64, or 32 for a short last
// chunk).  rowscale[n] = 2^(e_n) (N entries), colscale[k] = 2^(f_k) (kt
// entries; 1 in the padding).
size_t m2l_tc16_operator_halves(int p) { return (size_t)343 * 2 * m2l_rows(p) * tc_k(p); }

void pack_m2l_tc16_operators(int p, const double *m2l_in_major, uint16_t *out, float *rowscale,
                             float *colscale) {
  const int nc = ncoef(p), N = m2l_rows(p), kt = tc_k(p);
  const size_t nn = (size_t)nc * nc;
  auto T = [&](int code, int n, int k) { return m2l_in_major[code * nn + (size_t)k * nc + n]; };
  std::vector<int> e(nc, 0), f(nc, 0);
  auto cexp = [](double v) {  // smallest e with v <= 2^e (v > 0)
    int x = 0;
    const double m = std::frexp(v, &x);
    return m == 0.5 ? x - 1 : x;
  };
  for (int round = 0; round < 4; ++round) {
    for (int n = 0; n < nc; ++n) {
      double mx = 0.0;
      for (int code = 0; code < 343; ++code)
        for (int k = 0; k < nc; ++k) mx = std::max(mx, std::fabs(T(code, n, k)) * std::ldexp(1.0, -f[k]));
      e[n] = mx > 0.0 ? cexp(mx) : 0;
    }
    for (int k = 0; k < nc; ++k) {
      double mx = 0.0;
      for (int code = 0; code < 343; ++code)
        for (int n = 0; n < nc; ++n) mx = std::max(mx, std::fabs(T(code, n, k)) * std::ldexp(1.0, -e[n]));
      f[k] = mx > 0.0 ? cexp(mx) : 0;
    }
  }
  for (int n = 0; n < N; ++n) rowscale[n] = n < nc ? std::ldexp(1.0f, e[n]) : 1.0f;
  for (int k = 0; k < kt; ++k) colscale[k] = k < nc ? std::ldexp(1.0f, f[k]) : 1.0f;
  const int kt_bytes = 2 * kt, nch = (kt_bytes + kTcRowBytes - 1) / kTcRowBytes;
  for (int code = 0; code < 343; ++code)
    for (int c = 0; c < nch; ++c) {
      const int kc = std::min(kTcRowBytes, kt_bytes - c * kTcRowBytes) / 2;  // halves in this chunk
      uint16_t *hi = out + (size_t)code * 2 * N * kt + (size_t)c * 2 * N * (kTcRowBytes / 2);
      uint16_t *lo = hi + (size_t)N * kc;
      for (int n = 0; n < N; ++n)
        for (int kl = 0; kl < kc; ++kl) {
          const int k = c * (kTcRowBytes / 2) + kl;
          const float v = (n < nc && k < nc)
                              ? (float)(T(code, n, k) * std::ldexp(1.0, -e[n] - f[k]))
                              : 0.f;
          const __half h = __float2half_rn(v);
          const __half l = __float2half_rn(v - __half2float(h));
          // core matrices of 8 rows x 16 bytes; next along K 128 bytes on,
          // next along N (kc / 8) x 128 bytes on
          const size_t o = ((size_t)(n / 8) * (kc / 8) * 128 + (size_t)(kl / 8) * 128 + (n % 8) * 16 +
                            (kl % 8) * 2) / 2;
          hi[o] = __half_as_ushort(h);
          lo[o] = __half_as_ushort(l);
        }
    }
}

void launch_m2l_tc(int p, int64_t ntiles, const M2LTile *tiles, const int32_t *table,
                   const int16_t *slots, const int32_t *nslots, const int32_t *order, int64_t nb,
                   const float *M, const M2LTcForm &form, float *L, int *err, cudaStream_t s) {
  if (ntiles == 0) return;
  const int nc = ncoef(p), ld = coef_pitch(p), kt = tc_k(p), N = m2l_rows(p);
  const bool f16 = form.f16;
  if (f16) {
    k_split_f16<<<ceil_div(nb * 32, 256), 256, 0, s>>>(nb, nc, ld, kt, M, form.colscale,
                                                        reinterpret_cast<__half *>(form.Mhi),
                                                        reinterpret_cast<__half *>(form.Mlo),
                                                        form.mscale);
  } else {
    k_split_tf32<<<ceil_div(nb * kt, 256), 256, 0, s>>>(nb, nc, ld, kt, M,
                                                         reinterpret_cast<float *>(form.Mhi),
                                                         reinterpret_cast<float *>(form.Mlo));
  }
  FMM_LAUNCH_CHECK();
  // four stages where they fit in the 227 KB of shared memory per CTA, else three
  auto run = [&](auto NC, auto F) {
    constexpr int NTT = decltype(NC)::value;
    constexpr bool kF16 = decltype(F)::value;
    constexpr size_t stage = (size_t)2 * (kTcTile + NTT) * kTcRowBytes;
    constexpr int kStages = 4 * stage + 1024 + 512 <= 227 * 1024 ? 4 : 3;
    const size_t smem = kStages * stage + 1024;  // + alignment slack
    auto kern = k_m2l_tc<NTT, kStages, kF16>;
    FMM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)ntiles, kTcThreads, smem, s>>>(
        p, kt, tiles, table, slots, nslots, order,
        reinterpret_cast<const unsigned char *>(form.Mhi),
        reinterpret_cast<const unsigned char *>(form.Mlo),
        reinterpret_cast<const unsigned char *>(form.opt), form.mscale, form.rowscale, L, err);
  };
  auto run_n = [&](auto F) {
    switch (N) {
      case 16: run(std::integral_constant<int, 16>(), F); break;
      case 32: run(std::integral_constant<int, 32>(), F); break;
      case 48: run(std::integral_constant<int, 48>(), F); break;
      case 64: run(std::integral_constant<int, 64>(), F); break;
      case 96: run(std::integral_constant<int, 96>(), F); break;
      case 112: run(std::integral_constant<int, 112>(), F); break;
      case 128: run(std::integral_constant<int, 128>(), F); break;
      default: throw Error(FMM_ERR_UNSUPPORTED, "tensor-core M2L: unsupported operator size");
    }
  };
  if (f16) run_n(std::true_type());
  else run_n(std::false_type());
  FMM_LAUNCH_CHECK();
}

}  // namespace fmm

// tc_probe.cu -- self-check of the tensor-core path used by the M2L
// contraction: one CTA computes D[128][N] = A[128][K] B[N][K]^T with
// tcgen05.mma (kind::tf32, accumulator in tensor memory), either as one TF32
// product or as the three-product split (A_hi B_hi + A_hi B_lo + A_lo B_hi)
// that carries FP32 accuracy.  The operands use the layouts of the M2L
// kernel: A in 128-byte-swizzle tiles of 32 K values, B without swizzle.
// Every wait is bounded; a timeout is reported.
#include "plan.cuh"
#include "tcgen05.cuh"

namespace fmm {

namespace {

constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

__global__ void __launch_bounds__(128)
    k_tc_probe(int N, int K, const float *__restrict__ A, const float *__restrict__ B,
               float *__restrict__ D, int mode, int *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // swizzled tiles need a 1024-byte-aligned base (1 KB of slack is allocated)
  unsigned char *sm = sm_raw + ((1024u - (tc::smem_addr(sm_raw) & 1023u)) & 1023u);
  const int Kp = (K + 31) / 32 * 32;
  unsigned char *Ahi = sm, *Alo = Ahi + 128 * Kp * 4, *Bhi = Alo + 128 * Kp * 4, *Blo = Bhi + N * K * 4;
  for (int e = tid; e < 128 * K; e += 128) {
    const int r = e / K, k = e - r * K;
    float hi, lo;
    tc::split_tf32(A[e], hi, lo);
    const uint32_t o = (uint32_t)(k / 32) * 128 * 128 + tc::sw128_offset(r, k % 32);
    *reinterpret_cast<float *>(Ahi + o) = hi;
    *reinterpret_cast<float *>(Alo + o) = lo;
  }
  for (int e = tid; e < N * K; e += 128) {
    const int r = e / K, k = e - r * K;
    float hi, lo;
    tc::split_tf32(B[e], hi, lo);
    *reinterpret_cast<float *>(Bhi + tc::kmajor_offset(r, k, K)) = hi;
    *reinterpret_cast<float *>(Blo + tc::kmajor_offset(r, k, K)) = lo;
  }
  const uint32_t ncols = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  tc::fence_async_shared();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_tf32(128, N);
    const uint32_t sbo = (uint32_t)(K / 4) * 128;
    for (int ks = 0; ks < K / 8; ++ks) {
      const uint32_t off = (uint32_t)ks * 256;
      const uint32_t aoff = (uint32_t)(ks / 4) * 128 * 128 + (uint32_t)(ks % 4) * 32;
      const uint64_t ah = tc::smem_desc_sw128(tc::smem_addr(Ahi) + aoff);
      const uint64_t al = tc::smem_desc_sw128(tc::smem_addr(Alo) + aoff);
      const uint64_t bh = tc::smem_desc(tc::smem_addr(Bhi) + off, 128, sbo);
      const uint64_t bl = tc::smem_desc(tc::smem_addr(Blo) + off, 128, sbo);
      tc::mma_tf32(tmem, ah, bh, idesc, ks > 0);
      if (mode == 3) {
        tc::mma_tf32(tmem, ah, bl, idesc, 1);
        tc::mma_tf32(tmem, al, bh, idesc, 1);
      }
    }
    tc::mma_commit(&mbar);
  }
  bool ok = tc::mbar_wait_bounded(&mbar, 0, kWaitCycles);
  if (!ok) {
    if (lane == 0) atomicExch(err, 1);
    ok = tc::mbar_wait_bounded(&mbar, 0, kWaitCycles);  // give in-flight MMAs a second chance
  }
  tc::fence_after_sync();
  if (ok) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      for (int i = 0; i < 16 && c0 + i < N; ++i) D[(warp * 32 + lane) * N + c0 + i] = v[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// The bounded wait of the tensor-core kernels, on an mbarrier of one expected
// arrival: with arrive != 0 the thread arrives first and the wait completes;
// with arrive == 0 nothing arrives, the wait gives up after limit cycles and
// the kernel records that in err and returns (no trap, no endless loop).
__global__ void k_wait_probe(int arrive, long long limit, int *__restrict__ err) {
  __shared__ uint64_t mbar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&mbar, 1);
  if (arrive) tc::mbar_arrive(&mbar);
  if (!tc::mbar_wait_bounded(&mbar, 0, limit)) *err = 1;
}

}  // namespace

}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_wait_selftest(int arrive, long long limit_cycles, void *stream) {
  if (limit_cycles < 1 || limit_cycles > kWaitCycles)
    return record_error(FMM_ERR_INVALID_ARG, "fmm_wait_selftest: limit_cycles in 1..2e9");
  try {
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<int> err;
    err.resize(1, s);
    FMM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_wait_probe<<<1, 32, 0, s>>>(arrive, limit_cycles, err.p);
    FMM_LAUNCH_CHECK();
    int h = 0;
    FMM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    err.release();
    if (h) return record_error(FMM_ERR_TIMEOUT, "wait probe: the bounded mbarrier wait gave up");
    return FMM_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  }
}

extern "C" fmm_status fmm_tc_selftest(int n, int k, const float *d_a, const float *d_b, float *d_d,
                                      int mode, void *stream) {
  if (n < 16 || n > 256 || n % 16 != 0 || k < 8 || k % 8 != 0 || (mode != 1 && mode != 3) ||
      !d_a || !d_b || !d_d)
    return record_error(FMM_ERR_INVALID_ARG,
                        "fmm_tc_selftest: n in 16..256 (multiple of 16), k multiple of 8, mode 1 or 3");
  const size_t kp = (size_t)(k + 31) / 32 * 32;
  const size_t smem = (2 * 128 * kp + 2 * (size_t)n * k) * sizeof(float) + 1024;
  if (smem > 201 * 1024) return record_error(FMM_ERR_INVALID_ARG, "fmm_tc_selftest: operands too large");
  try {
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<int> err;
    err.resize(1, s);
    FMM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    FMM_CUDA(cudaFuncSetAttribute(k_tc_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tc_probe<<<1, 128, smem, s>>>(n, k, d_a, d_b, d_d, mode, err.p);
    FMM_LAUNCH_CHECK();
    int h = 0;
    FMM_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    err.release();
    if (h) return record_error(FMM_ERR_TIMEOUT, "tensor-core probe: MMA completion wait timed out");
    return FMM_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  }
}

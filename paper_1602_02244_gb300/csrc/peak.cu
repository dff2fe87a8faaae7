// peak.cu -- measured FP32 and FP64 rates of this GPU, the denominators of
// the rooflines of the FP32-bound passes (P2P, and the CUDA-core M2L path)
// and of the FP64-bound ones (the Helmholtz translations and near field).  A
// grid that fills every SM runs independent chains of fused multiply-adds:
// paired for FP32 (fma.rn.f32x2, two FMAs per lane and instruction, as the
// P2P kernel issues them), plain for FP64; achieved = 2 flop x FMAs / time,
// best over a few launch shapes.
#include <algorithm>

#include "plan.cuh"

namespace fmm {

namespace {

template <int CHAINS>
__global__ void k_fp32_peak(int iters, float seed, float *__restrict__ sink) {
  float2 a[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) a[i] = make_float2(seed * (threadIdx.x + i), seed * i);
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = __ffma2_rn(a[i], m, c);
  }
  float v = 0.f;
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) v += a[i].x + a[i].y;
  if (v == -1.f) sink[0] = v;  // keeps the chains live; never true for these inputs
}

template <int CHAINS>
__global__ void k_fp64_peak(int iters, double seed, double *__restrict__ sink) {
  double a[CHAINS];
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) a[i] = seed * (threadIdx.x + i);
  const double m = 0.9999999999, c = 1e-15;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CHAINS; ++i) a[i] = fma(a[i], m, c);
  }
  double v = 0.0;
#pragma unroll
  for (int i = 0; i < CHAINS; ++i) v += a[i];
  if (v == -1.0) sink[0] = v;  // keeps the chains live; never true for these inputs
}

}  // namespace

// Best FP64 rate over a few shapes, as measure_fp32_peak below.
double measure_fp64_peak(cudaStream_t s) {
  int dev = 0, sms = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  FMM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBuf<double> sink;
  sink.resize(1, s);
  cudaEvent_t a = nullptr, b = nullptr;
  double best = 0.0;
  auto shape = [&](auto kern, int chains, int threads) {
    int per_sm = 0;
    FMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 2048 / chains;
    kern<<<grid, threads, 0, s>>>(16, 1e-3, sink.p);  // warm-up
    FMM_LAUNCH_CHECK();
    for (int rep = 0; rep < 5; ++rep) {
      FMM_CUDA(cudaEventRecord(a, s));
      kern<<<grid, threads, 0, s>>>(iters, 1e-3, sink.p);
      FMM_LAUNCH_CHECK();
      FMM_CUDA(cudaEventRecord(b, s));
      FMM_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      FMM_CUDA(cudaEventElapsedTime(&ms, a, b));
      const double flop = 2.0 * chains * (double)iters * threads * grid;
      if (ms > 0.f) best = std::max(best, flop / (ms * 1e-3));
    }
  };
  try {
    FMM_CUDA(cudaEventCreate(&a));
    FMM_CUDA(cudaEventCreate(&b));
    shape(k_fp64_peak<8>, 8, 256);
    shape(k_fp64_peak<8>, 8, 512);
    shape(k_fp64_peak<16>, 16, 256);
    shape(k_fp64_peak<16>, 16, 512);
  } catch (...) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    sink.release();
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  sink.release();
  return best;
}

// Best rate over a few shapes (independent chains per thread x threads per
// block, every SM filled to its occupancy), each timed over five launches of
// about a millisecond: the attainable FP32 rate, not one shape's.
double measure_fp32_peak(cudaStream_t s) {
  int dev = 0, sms = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  FMM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBuf<float> sink;
  sink.resize(1, s);
  cudaEvent_t a = nullptr, b = nullptr;
  double best = 0.0;
  auto shape = [&](auto kern, int chains, int threads) {
    int per_sm = 0;
    FMM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 32768 / chains;  // the same work per thread for every shape
    kern<<<grid, threads, 0, s>>>(64, 1e-3f, sink.p);  // warm-up
    FMM_LAUNCH_CHECK();
    for (int rep = 0; rep < 5; ++rep) {
      FMM_CUDA(cudaEventRecord(a, s));
      kern<<<grid, threads, 0, s>>>(iters, 1e-3f, sink.p);
      FMM_LAUNCH_CHECK();
      FMM_CUDA(cudaEventRecord(b, s));
      FMM_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      FMM_CUDA(cudaEventElapsedTime(&ms, a, b));
      const double flop = 4.0 * chains * (double)iters * threads * grid;  // 2 lanes x 2 flop
      if (ms > 0.f) best = std::max(best, flop / (ms * 1e-3));
    }
  };
  try {
    FMM_CUDA(cudaEventCreate(&a));
    FMM_CUDA(cudaEventCreate(&b));
    shape(k_fp32_peak<8>, 8, 256);
    shape(k_fp32_peak<8>, 8, 512);
    shape(k_fp32_peak<16>, 16, 256);
    shape(k_fp32_peak<16>, 16, 512);
  } catch (...) {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    sink.release();
    throw;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  sink.release();
  return best;
}

}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_fp32_peak(double *tflops, void *stream) {
  if (!tflops) return record_error(FMM_ERR_INVALID_ARG, "fmm_fp32_peak: NULL output");
  try {
    *tflops = measure_fp32_peak((cudaStream_t)stream) / 1e12;
    return FMM_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  }
}

extern "C" fmm_status fmm_fp64_peak(double *tflops, void *stream) {
  if (!tflops) return record_error(FMM_ERR_INVALID_ARG, "fmm_fp64_peak: NULL output");
  try {
    *tflops = measure_fp64_peak((cudaStream_t)stream) / 1e12;
    return FMM_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  }
}

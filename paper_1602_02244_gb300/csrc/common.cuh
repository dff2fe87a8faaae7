// common.cuh -- shared device helpers and plan layout of libfmm (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/fmm.h"

namespace fmm {

constexpr int kMaxDepth = 21;  // 21 bits per axis, 63-bit Morton keys
constexpr int kMaxOrder = 20;

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
  fmm_status status;
  Error(fmm_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define FMM_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::fmm::Error(e_ == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

// every kernel launch is followed by FMM_LAUNCH_CHECK(), which also counts it
void note_launch();
#define FMM_LAUNCH_CHECK()             \
  do {                                 \
    ::fmm::note_launch();              \
    FMM_CUDA(cudaGetLastError());      \
  } while (0)

// sets the message returned by fmm_last_error_message() and returns s
fmm_status record_error(fmm_status s, const std::string &msg);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------- device buffers
// Stream-ordered allocations from a library-owned memory pool that keeps
// its memory between plans (no cudaMalloc after the first plan of a size).
void *device_alloc(size_t bytes, cudaStream_t s);
void device_free(void *p, cudaStream_t s);

template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0, cap = 0;
  cudaStream_t s = nullptr;
  // (re)size to exactly n elements; contents are not preserved
  void resize(size_t count, cudaStream_t st) {
    s = st;
    if (count > cap) {
      if (p) device_free(p, st);
      size_t c = count + count / 8 + 64;
      p = (T *)device_alloc(c * sizeof(T), st);
      cap = c;
    }
    n = count;
  }
  // grow keeping the first `keep` elements
  void grow(size_t count, size_t keep, cudaStream_t st) {
    s = st;
    if (count > cap) {
      size_t c = count + count / 2 + 64;
      T *q = (T *)device_alloc(c * sizeof(T), st);
      if (p && keep) FMM_CUDA(cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, st));
      if (p) device_free(p, st);
      p = q;
      cap = c;
    }
    n = count;
  }
  void release() {
    if (p) device_free(p, s);
    p = nullptr;
    n = cap = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------- morton bits
__host__ __device__ inline uint64_t spread3(uint32_t v) {
  // place bit b of v (b < 21) at bit 3b
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__host__ __device__ inline uint32_t compact3(uint64_t x) {
  // inverse of spread3
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x1f00000000ffffull;
  x = (x | (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

__host__ __device__ inline uint64_t morton3(uint32_t ix, uint32_t iy, uint32_t iz) {
  return spread3(ix) | (spread3(iy) << 1) | (spread3(iz) << 2);
}

// --------------------------------------------------------- coefficients
__host__ __device__ constexpr int ncoef(int p) { return (p + 1) * (p + 1); }
__host__ __device__ constexpr int cidx(int n, int m) { return n * n + n + m; }
// row pitch (in elements) of coefficient arrays and padded operators: a
// multiple of 4 (16-byte rows for FP32) whose quarter is odd, so rows read as
// float4 by consecutive threads fall in distinct shared-memory bank groups
__host__ __device__ constexpr int coef_pitch(int p) {
  return ((ncoef(p) + 3) / 4 % 2 == 1) ? (ncoef(p) + 3) / 4 * 4 : (ncoef(p) + 3) / 4 * 4 + 4;
}

// Box geometry record: integer anchor at its level and the level.
// four doubles on a 32-byte boundary (one point or one per-target record)
struct __align__(32) Dbl4 {
  double x, y, z, w;
};
__host__ __device__ __forceinline__ Dbl4 make_dbl4(double x, double y, double z, double w) {
  Dbl4 v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = w;
  return v;
}

// Sort a short run of box numbers in place (Shell sort with Ciura's gaps;
// plain insertion for runs up to 32).
__device__ inline void sort_run(int32_t *a, int n) {
  const int gaps[] = {301, 132, 57, 23, 10, 4, 1};
  for (int gi = 0; gi < 7; ++gi) {
    const int gap = gaps[gi];
    if (gap >= n) continue;
    for (int i = gap; i < n; ++i) {
      const int32_t v = a[i];
      int j = i;
      while (j >= gap && a[j - gap] > v) {
        a[j] = a[j - gap];
        j -= gap;
      }
      a[j] = v;
    }
  }
}

struct __align__(16) BoxGeo {
  int32_t ix, iy, iz, level;
};

// side length of a box at level l of a root cube of side D
__host__ __device__ inline double box_side(double D, int l) { return ldexp(D, -l); }

}  // namespace fmm

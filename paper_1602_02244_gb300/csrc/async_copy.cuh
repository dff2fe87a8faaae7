// async_copy.cuh -- 16-byte asynchronous global-to-shared copies (cp.async,
// sm_80 and later), grouped and waited on per thread.  A copy is visible to
// the other threads of the block after cp_async_wait and a barrier.
#pragma once
#include <cstdint>

namespace fmm {

// copies src_bytes (0 or 16) from gmem and zero-fills the rest of the 16 bytes
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace fmm

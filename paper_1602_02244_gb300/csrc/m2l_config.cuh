// m2l_config.cuh -- tile shapes of the per-level M2L kernel.
//
// A CTA owns TILE target boxes of one level that share their octant parity,
// so every target's interaction-list offsets fall on one 6x6x6 slot grid
// (§2.2: children of the parent's colleagues, at most 189 of the 216).  For
// each occupied slot it stages the slot's translation matrix and the
// targets' source multipoles through shared memory and accumulates
// L[target] += T(offset) M[source] in registers (TPT targets x RPT rows per
// thread, 256 threads).
#pragma once
#include "common.cuh"

namespace fmm {

constexpr int kM2LThreads = 256;
constexpr int kM2LKC = 16;  // k-chunk of the contraction staged per step

struct M2LShape {
  int tile, tpt, rpt;
};

inline M2LShape m2l_shape(int order) {
  int nc = ncoef(order);
  if (nc <= 128) {
    int rpt = (nc + 15) / 16;
    if (rpt == 5) rpt = 6;  // instantiated row counts: 1,2,3,4,6,7,8
    return {64, 4, rpt};
  }
  if (nc <= 256) return {32, 2, 16};
  return {16, 1, 28};
}

inline int m2l_tile_size(int order, int /*precision*/) { return m2l_shape(order).tile; }
constexpr int kM2LTensorTile = 128;  // targets per CTA of the tensor-core path (MMA M)

// Staged FP32 kernel (orders up to 10): 64 targets x 16*RPT rows per CTA,
// one whole slot (operator + gathered multipoles) per pipeline stage.
constexpr int kM2LStagedMaxOrder = 10;
// rotated M2L: orders whose rotation tables are built at plan time
constexpr int kRotMaxOrder = 12;
__host__ __device__ constexpr int m2l_rows(int order) { return (ncoef(order) + 15) / 16 * 16; }

}  // namespace fmm

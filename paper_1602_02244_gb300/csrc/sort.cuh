// sort.cuh -- device-wide exclusive scan and stable LSD radix sort.
#pragma once
#include "common.cuh"

namespace fmm {

// out[i] = sum_{j<i} in[i]; if d_total != nullptr, *d_total = sum of all.
// in and out may alias.  `tmp` is resized as needed.
void scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total,
                    DBuf<int32_t> &tmp, cudaStream_t s);

// Stable sort of (keys, vals) by the key bits in the listed 8-bit digit
// shifts (processed in the given order, least significant first).  vals may
// be absent (vals.p == nullptr).  Results end up in keys/vals (the DBufs are
// swapped with the temporaries as the passes go).
void radix_sort(DBuf<uint64_t> &keys, DBuf<int32_t> &vals, DBuf<uint64_t> &tkeys,
                DBuf<int32_t> &tvals, int64_t n, const std::vector<int> &shifts,
                DBuf<int32_t> &hist, DBuf<int32_t> &tmp, cudaStream_t s);

// digit shifts covering bits [lo, hi)
std::vector<int> digit_shifts(int lo, int hi);

}  // namespace fmm

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

// Raw-pointer variants for callers that bring their own scratch memory.
// scan: block_sums holds scan_raw_tmp_elems(n) ints.  radix sort: an even
// number of passes leaves the result in keys/vals; hist holds
// radix_raw_hist_elems(n) ints and scan_tmp scan_raw_tmp_elems(that) ints.
size_t scan_raw_tmp_elems(int64_t n);
size_t radix_raw_hist_elems(int64_t n);
void scan_exclusive_raw(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total,
                        int32_t *block_sums, cudaStream_t s);
void radix_sort_raw(uint64_t *keys, int32_t *vals, uint64_t *tkeys, int32_t *tvals, int64_t n,
                    const int *shifts, int nshifts, int32_t *hist, int32_t *scan_tmp,
                    cudaStream_t s);

// digit shifts covering bits [lo, hi)
std::vector<int> digit_shifts(int lo, int hi);

}  // namespace fmm

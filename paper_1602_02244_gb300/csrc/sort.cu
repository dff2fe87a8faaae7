// sort.cu -- exclusive scan and stable LSD radix sort for sm_103a.
//
// Radix sort: reduce-then-scan per 8-bit digit.  (1) every CTA counts the
// digits of its 4096-key tile; (2) one device-wide exclusive scan over the
// digit-major count table gives every (digit, tile) its output base; (3) every
// CTA ranks its keys stably (warp match_any per 32-key round, warp-ordered
// digit counters in shared memory), stages the tile in shared memory in digit
// order and writes each digit's run contiguously.  No inter-CTA waits.
#include "sort.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace fmm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *warp_sums,
                                                        int32_t *total) {
  // exclusive scan of one value per thread across a 256-thread block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < (kScanThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kScanThreads / 32)) warp_sums[lane] = w;  // inclusive
  }
  __syncthreads();
  int32_t base = warp > 0 ? warp_sums[warp - 1] : 0;
  if (total) *total = warp_sums[kScanThreads / 32 - 1];
  return base + x - v;
}

__global__ void k_scan_reduce(const int32_t *__restrict__ in, int64_t n, int32_t *sums) {
  __shared__ int32_t ws[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int32_t tot;
  block_exclusive_scan(s, ws, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t *sums, int nblocks, int32_t *d_total) {
  // single CTA: exclusive scan of the block sums in chunks of 256
  __shared__ int32_t ws[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c = 0; c < nblocks; c += kScanThreads) {
    int i = c + threadIdx.x;
    int32_t v = i < nblocks ? sums[i] : 0;
    int32_t tot;
    int32_t ex = block_exclusive_scan(v, ws, &tot);
    int32_t base = carry;
    if (i < nblocks) sums[i] = base + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry = base + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

// Small inputs: one CTA walks the array in tiles of kScanTile with a running
// carry -- one launch instead of three (in place is allowed).
constexpr int64_t kScanSingleMax = 16384;

__global__ void k_scan_single(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total) {
  __shared__ int32_t ws[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t t0 = 0; t0 < n; t0 += kScanTile) {
    const int64_t base = t0 + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = base + k < n ? in[base + k] : 0;
      sum += v[k];
    }
    int32_t tot;
    int32_t ex = block_exclusive_scan(sum, ws, &tot) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      if (base + k < n) out[base + k] = ex;
      ex += v[k];
    }
    __syncthreads();  // everyone has read carry
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void k_scan_apply(const int32_t *in, int32_t *out, int64_t n, const int32_t *sums) {
  // each thread owns kScanItems consecutive elements of the tile
  __shared__ int32_t ws[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int32_t ex = block_exclusive_scan(s, ws, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
}

// ------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsTile = kRsThreads * kRsItems;  // 4096 keys per CTA
constexpr int kRsWarpSeg = 32 * kRsItems;       // 512 keys per warp
constexpr int kRsSmemKeys = kRsTile * 8;        // staged tile: keys
constexpr int kRsSmemVals = kRsTile * 12;       // keys and 32-bit values

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             int32_t *__restrict__ hist, int nblocks) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int k = 0; k < kRsItems; ++k) {
    int64_t i = base + (int64_t)k * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter one 8-bit digit pass.  Each warp ranks its 512 keys per digit
// (match_any), the CTA turns the per-warp counts into tile-local digit
// offsets, places its 4096 keys in shared memory in digit order, and then
// writes each digit's run to its global slot with consecutive threads on
// consecutive addresses.  The order within a digit is (warp, item, lane),
// i.e. input order: the sort is stable.
template <bool kVals>
__global__ void __launch_bounds__(kRsThreads)
    k_radix_scatter(const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, int64_t n,
                    int shift, const int32_t *__restrict__ offs, int nblocks,
                    uint64_t *__restrict__ kout, int32_t *__restrict__ vout) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(rs_smem);  // kRsTile keys
  int32_t *sv = reinterpret_cast<int32_t *>(sk + kRsTile);  // kRsTile values
  __shared__ int32_t whist[kRsWarps][256];
  __shared__ int32_t gbase[256], dstart[256], wsum[kRsWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < kRsWarps; ++w) whist[w][threadIdx.x] = 0;
  gbase[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t tile0 = (int64_t)blockIdx.x * kRsTile;
  const int64_t seg = tile0 + (int64_t)warp * kRsWarpSeg;
  uint64_t key[kRsItems];
  int32_t val[kRsItems];
  int32_t rank[kRsItems];
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    int64_t i = seg + r * 32 + lane;
    bool valid = i < n;
    key[r] = valid ? kin[i] : 0;
    if (kVals) val[r] = valid ? vin[i] : 0;
    unsigned d = valid ? (unsigned)((key[r] >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int32_t prev = valid ? whist[warp][d] : 0;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) whist[warp][d] = prev + __popc(peers);
    __syncwarp();
    rank[r] = prev + __popc(peers & lt_mask);
  }
  __syncthreads();
  {  // per digit (thread = digit): exclusive scan over warps, then over digits
    int32_t tot = 0;
    for (int w = 0; w < kRsWarps; ++w) {
      int32_t c = whist[w][threadIdx.x];
      whist[w][threadIdx.x] = tot;
      tot += c;
    }
    int32_t v = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    int32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    dstart[threadIdx.x] = woff + v - tot;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsItems; ++r) {
    int64_t i = seg + r * 32 + lane;
    if (i < n) {
      unsigned d = (unsigned)((key[r] >> shift) & 255u);
      const int32_t lp = dstart[d] + whist[warp][d] + rank[r];
      sk[lp] = key[r];
      if (kVals) sv[lp] = val[r];
    }
  }
  __syncthreads();
  const int cnt = (int)min((int64_t)kRsTile, n - tile0);
  for (int i = threadIdx.x; i < cnt; i += kRsThreads) {
    const uint64_t k = sk[i];
    const unsigned d = (unsigned)((k >> shift) & 255u);
    const int64_t pos = (int64_t)gbase[d] + (i - dstart[d]);
    kout[pos] = k;
    if (kVals) vout[pos] = sv[i];
  }
}

}  // namespace

void scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total,
                    DBuf<int32_t> &tmp, cudaStream_t s) {
  if (n <= 0) {
    if (d_total) FMM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int32_t), s));
    return;
  }
  if (n <= kScanSingleMax) {
    k_scan_single<<<1, kScanThreads, 0, s>>>(in, out, n, d_total);
    FMM_LAUNCH_CHECK();
    return;
  }
  int nb = ceil_div(n, kScanTile);
  tmp.resize(nb, s);
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, tmp.p);
  FMM_LAUNCH_CHECK();
  k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp.p, nb, d_total);
  FMM_LAUNCH_CHECK();
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, tmp.p);
  FMM_LAUNCH_CHECK();
}

size_t scan_raw_tmp_elems(int64_t n) { return n > 0 ? (size_t)ceil_div(n, kScanTile) : 1; }

size_t radix_raw_hist_elems(int64_t n) { return (size_t)256 * (n > 0 ? ceil_div(n, kRsTile) : 1); }

void scan_exclusive_raw(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total,
                        int32_t *block_sums, cudaStream_t s) {
  if (n <= 0) {
    if (d_total) FMM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int32_t), s));
    return;
  }
  int nb = ceil_div(n, kScanTile);
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, block_sums);
  FMM_LAUNCH_CHECK();
  k_scan_sums<<<1, kScanThreads, 0, s>>>(block_sums, nb, d_total);
  FMM_LAUNCH_CHECK();
  k_scan_apply<<<nb, kScanThreads, 0, s>>>(in, out, n, block_sums);
  FMM_LAUNCH_CHECK();
}

// The staged scatter needs more than the default 48 KB of dynamic shared
// memory; the opt-in is set once per device.
static void launch_scatter(const uint64_t *keys, const int32_t *vals, int64_t n, int sh,
                    const int32_t *hist, int nb, uint64_t *tkeys, int32_t *tvals, cudaStream_t s) {
  static std::mutex mu;
  static std::vector<int> configured;
  int dev = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(configured.begin(), configured.end(), dev) == configured.end()) {
      FMM_CUDA(cudaFuncSetAttribute(k_radix_scatter<true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kRsSmemVals));
      FMM_CUDA(cudaFuncSetAttribute(k_radix_scatter<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, kRsSmemKeys));
      configured.push_back(dev);
    }
  }
  if (vals)
    k_radix_scatter<true><<<nb, kRsThreads, kRsSmemVals, s>>>(keys, vals, n, sh, hist, nb, tkeys,
                                                               tvals);
  else
    k_radix_scatter<false><<<nb, kRsThreads, kRsSmemKeys, s>>>(keys, nullptr, n, sh, hist, nb,
                                                                tkeys, nullptr);
  FMM_LAUNCH_CHECK();
}

void radix_sort_raw(uint64_t *keys, int32_t *vals, uint64_t *tkeys, int32_t *tvals, int64_t n,
                    const int *shifts, int nshifts, int32_t *hist, int32_t *scan_tmp,
                    cudaStream_t s) {
  if (n <= 1 || nshifts <= 0) return;
  if (nshifts % 2 != 0) throw Error(FMM_ERR_INVALID_ARG, "radix_sort_raw needs an even pass count");

  int nb = ceil_div(n, kRsTile);
  for (int ip = 0; ip < nshifts; ++ip) {
    const int sh = shifts[ip];
    k_radix_hist<<<nb, kRsThreads, 0, s>>>(keys, n, sh, hist, nb);
    FMM_LAUNCH_CHECK();
    scan_exclusive_raw(hist, hist, (int64_t)256 * nb, nullptr, scan_tmp, s);
    launch_scatter(keys, vals, n, sh, hist, nb, tkeys, tvals, s);
    std::swap(keys, tkeys);
    std::swap(vals, tvals);
  }
}

std::vector<int> digit_shifts(int lo, int hi) {
  std::vector<int> v;
  for (int b = lo; b < hi; b += 8) v.push_back(b);
  return v;
}

void radix_sort(DBuf<uint64_t> &keys, DBuf<int32_t> &vals, DBuf<uint64_t> &tkeys,
                DBuf<int32_t> &tvals, int64_t n, const std::vector<int> &shifts,
                DBuf<int32_t> &hist, DBuf<int32_t> &tmp, cudaStream_t s) {
  if (n <= 1 || shifts.empty()) return;
  const bool has_vals = vals.p != nullptr;
  int nb = ceil_div(n, kRsTile);
  hist.resize((size_t)256 * nb, s);
  tkeys.resize(n, s);
  if (has_vals) tvals.resize(n, s);
  for (int sh : shifts) {
    k_radix_hist<<<nb, kRsThreads, 0, s>>>(keys.p, n, sh, hist.p, nb);
    FMM_LAUNCH_CHECK();
    scan_exclusive(hist.p, hist.p, (int64_t)256 * nb, nullptr, tmp, s);
    launch_scatter(keys.p, has_vals ? vals.p : nullptr, n, sh, hist.p, nb, tkeys.p,
                   has_vals ? tvals.p : nullptr, s);
    std::swap(keys, tkeys);
    if (has_vals) std::swap(vals, tvals);
  }
}

}  // namespace fmm

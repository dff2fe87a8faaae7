// noalloc.cu -- Morton keys and their stable sort without any device
// allocation.
//
// Some callers cannot let a library call cudaMalloc: a host application
// whose memory manager has already reserved all free device memory for its
// own pool, or a latency-critical loop that forbids cudaMalloc/cudaFree
// because those calls can synchronise the device and take unbounded time.
// fmm_morton_sort_noalloc serves them: it runs the same root-cube, Morton
// and radix-sort kernels as fmm_plan_create, but its scratch memory is a
// fixed array of this file, reserved on every GPU that loads the library
// and held until the process exits.  The caller provides the inputs and
// outputs.
#include <mutex>
#include <vector>

#include "plan.cuh"
#include "sort.cuh"

namespace fmm {

namespace {

constexpr int64_t kNoAllocMaxPoints = FMM_NOALLOC_MAX_POINTS;
constexpr int kMaxDevices = 64;

// scratch layout (byte offsets, all 256-byte aligned)
constexpr size_t kTmpKeysOff = 0;
constexpr size_t kTmpKeysBytes = 8 * (size_t)kNoAllocMaxPoints;
constexpr size_t kTmpValsOff = kTmpKeysOff + kTmpKeysBytes;
constexpr size_t kTmpValsBytes = 4 * (size_t)kNoAllocMaxPoints;
constexpr size_t kHistOff = kTmpValsOff + kTmpValsBytes;
constexpr size_t kHistElems = 256 * (size_t)((kNoAllocMaxPoints + 4095) / 4096);
constexpr size_t kHistBytes = 4 * kHistElems;
constexpr size_t kScanOff = kHistOff + kHistBytes;
constexpr size_t kScanBytes = 4 * 1024;  // >= ceil(kHistElems / 2048) block sums
constexpr size_t kPartialOff = kScanOff + kScanBytes;
constexpr size_t kPartialBytes = 8 * 7 * 1024;
constexpr size_t kGeomOff = kPartialOff + kPartialBytes;
constexpr size_t kGeomBytes = 256;
constexpr size_t kScratchBytes = kGeomOff + kGeomBytes;
static_assert(kHistOff % 256 == 0 && kScanOff % 256 == 0 && kPartialOff % 256 == 0 &&
                  kGeomOff % 256 == 0,
              "scratch sub-buffers must stay aligned");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: kernels must be given the device address from
// cudaGetSymbolAddress, looked up once per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// The radix passes: the digits of a Morton key (3 bits per level), padded to
// an even pass count so that the sorted result ends in the caller's arrays.
constexpr int kKeyBits = 3 * kMaxDepth;
constexpr int kPasses = ((kKeyBits + 7) / 8 + 1) / 2 * 2;
static_assert(kPasses == 8, "the 63-bit keys take eight 8-bit passes");

unsigned char *scratch_for_device(cudaStream_t s) {
  int dev = 0;
  FMM_CUDA(cudaGetDevice(&dev));
  if (s) {  // a stream of another device would run the kernels against that device's array
    int sdev = dev;
    FMM_CUDA(cudaStreamGetDevice(s, &sdev));
    if (sdev != dev)
      throw Error(FMM_ERR_INVALID_ARG,
                  "fmm_morton_sort_noalloc: the stream belongs to another device than the current one");
  }
  if (dev < 0 || dev >= kMaxDevices) throw Error(FMM_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      throw Error(FMM_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                    cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_morton_sort_noalloc(const double *d_xyz, int64_t n, uint64_t *d_keys,
                                              int32_t *d_perm, double *h_root, void *stream) {
  if (n < 0 || n > kNoAllocMaxPoints) {
    return record_error(FMM_ERR_INVALID_ARG,
                            "fmm_morton_sort_noalloc: n must be in [0, FMM_NOALLOC_MAX_POINTS = "
                            "1048576]; use fmm_plan_create for larger inputs");
  }
  if (n > 0 && (!d_xyz || !d_keys || !d_perm))
    return record_error(FMM_ERR_INVALID_ARG, "fmm_morton_sort_noalloc: a device pointer is NULL");
  try {
    cudaStream_t s = (cudaStream_t)stream;
    // the read-back below cannot be captured: refuse before touching the stream
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FMM_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
      return record_error(FMM_ERR_INVALID_ARG,
                          "fmm_morton_sort_noalloc: the stream is capturing a CUDA graph; every "
                          "call synchronises its stream and cannot be captured");
    unsigned char *base = scratch_for_device(s);
    if (n == 0) return FMM_OK;
    double *partial = reinterpret_cast<double *>(base + kPartialOff);
    double *geom = reinterpret_cast<double *>(base + kGeomOff);
    // every scratch word read below is written first in this call: the
    // histogram and scan kernels overwrite their whole range each pass
    morton_keys_raw(d_xyz, n, partial, geom, d_keys, d_perm, s);
    double hg[5];
    FMM_CUDA(cudaMemcpyAsync(hg, geom, sizeof hg, cudaMemcpyDeviceToHost, s));
    FMM_CUDA(cudaStreamSynchronize(s));
    if (hg[4] != 0.0)
      return record_error(FMM_ERR_NONFINITE_INPUT, "a coordinate is NaN or infinite");
    if (h_root)
      for (int a = 0; a < 4; ++a) h_root[a] = hg[a];
    // the plan's digit order (digit_shifts(0, 3 * kMaxDepth)), padded to kPasses
    std::vector<int> shifts = digit_shifts(0, kKeyBits);
    while ((int)shifts.size() < kPasses) shifts.push_back(shifts.back() + 8);
    radix_sort_raw(d_keys, d_perm, reinterpret_cast<uint64_t *>(base + kTmpKeysOff),
                   reinterpret_cast<int32_t *>(base + kTmpValsOff), n, shifts.data(), kPasses,
                   reinterpret_cast<int32_t *>(base + kHistOff),
                   reinterpret_cast<int32_t *>(base + kScanOff), s);
    return FMM_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  }
}

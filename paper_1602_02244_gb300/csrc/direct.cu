// direct.cu -- brute-force evaluation of the Laplace potential and its
// gradient, the plain definition the FMM approximates (§2, Eq. 1 with the
// 1/r kernel):
//   phi(t)  =  sum_{j : x_j != t} q_j / |t - x_j|,
//   grad(t) = -sum_{j : x_j != t} q_j (t - x_j) / |t - x_j|^3.
// FP64 throughout.  Sources are cut into chunks along grid.y; each CTA keeps
// 128 targets in registers, stages 256 sources at a time in shared memory and
// writes its partial sums; a second kernel adds the chunks in chunk order, so
// the result does not depend on scheduling.
#include "plan.cuh"

namespace fmm {

namespace {

constexpr int kDirThreads = 128;  // targets per CTA
constexpr int kDirTile = 256;     // sources staged per round

struct alignas(32) Src4 {
  double x, y, z, q;
};

__global__ void __launch_bounds__(kDirThreads)
    k_direct(const double *__restrict__ src, const double *__restrict__ q, int64_t n,
             const double *__restrict__ tgt, int64_t m, int64_t chunk, double *__restrict__ part) {
  __shared__ Src4 ss[kDirTile];
  const int64_t t = (int64_t)blockIdx.x * kDirThreads + threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(n, j0 + chunk);
  double x = 0, y = 0, z = 0;
  if (t < m) {
    x = tgt[3 * t];
    y = tgt[3 * t + 1];
    z = tgt[3 * t + 2];
  }
  double phi = 0, gx = 0, gy = 0, gz = 0;
  for (int64_t j = j0; j < j1; j += kDirTile) {
    const int cnt = (int)(j1 - j < kDirTile ? j1 - j : kDirTile);
    __syncthreads();  // the previous tile has been consumed
    for (int k = threadIdx.x; k < cnt; k += kDirThreads) {
      const int64_t g = j + k;
      ss[k] = Src4{src[3 * g], src[3 * g + 1], src[3 * g + 2], q[g]};
    }
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      const Src4 s = ss[k];
      const double dx = x - s.x, dy = y - s.y, dz = z - s.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 > 0) {  // coincident points contribute nothing
        const double rinv = 1.0 / sqrt(r2);
        const double qr = s.q * rinv, qr3 = qr * rinv * rinv;
        phi += qr;
        gx -= qr3 * dx;
        gy -= qr3 * dy;
        gz -= qr3 * dz;
      }
    }
  }
  if (t < m) {
    double *p = part + ((int64_t)blockIdx.y * m + t) * 4;
    p[0] = phi;
    p[1] = gx;
    p[2] = gy;
    p[3] = gz;
  }
}

__global__ void k_direct_sum(int64_t m, int nchunk, const double *__restrict__ part,
                             double *__restrict__ phi, double *__restrict__ grad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  for (int c = 0; c < nchunk; ++c) {
    const double *p = part + ((int64_t)c * m + t) * 4;
    a0 += p[0];
    a1 += p[1];
    a2 += p[2];
    a3 += p[3];
  }
  phi[t] = a0;
  if (grad) {
    grad[3 * t] = a1;
    grad[3 * t + 1] = a2;
    grad[3 * t + 2] = a3;
  }
}

}  // namespace

}  // namespace fmm

using namespace fmm;

extern "C" fmm_status fmm_direct(const double *d_src, const double *d_q, int64_t n,
                                 const double *d_tgt, int64_t m, double *d_phi, double *d_grad,
                                 void *stream) {
  if (n < 0 || m < 0) return record_error(FMM_ERR_INVALID_ARG, "fmm_direct: negative size");
  if (n > 0 && (!d_src || !d_q))
    return record_error(FMM_ERR_INVALID_ARG, "fmm_direct: d_src or d_q is NULL");
  if (m > 0 && (!d_tgt || !d_phi))
    return record_error(FMM_ERR_INVALID_ARG, "fmm_direct: d_tgt or d_phi is NULL");
  if (m == 0) return FMM_OK;
  DBuf<double> part;
  try {
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t tb = ceil_div(m, (int64_t)kDirThreads);
    // enough CTAs to fill the GPU twice over, each with at least 2048 sources
    int64_t nchunk = std::max<int64_t>(1, 2432 / tb);
    nchunk = std::min<int64_t>(nchunk, std::max<int64_t>(1, ceil_div(n, (int64_t)2048)));
    nchunk = std::min<int64_t>(nchunk, 65535);
    const int64_t chunk = n > 0 ? ceil_div(n, nchunk) : 0;
    part.resize((size_t)nchunk * m * 4, s);
    k_direct<<<dim3((unsigned)tb, (unsigned)nchunk), kDirThreads, 0, s>>>(d_src, d_q, n, d_tgt, m,
                                                                          chunk, part.p);
    FMM_LAUNCH_CHECK();
    k_direct_sum<<<(unsigned)ceil_div(m, (int64_t)256), 256, 0, s>>>(m, (int)nchunk, part.p, d_phi,
                                                                     d_grad);
    FMM_LAUNCH_CHECK();
    part.release();
    return FMM_OK;
  } catch (const Error &e) {
    try {
      part.release();
    } catch (const Error &) {
    }
    return record_error(e.status, e.what());
  }
}

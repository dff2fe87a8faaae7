// stencil.cu -- the 7-point discrete Laplacian on the interior of a cube with
// zero Dirichlet boundary values, and the Helmholtz operator built on it: the
// PDE operators of the paper's preconditioning experiment (§4.2), whose
// inverses the FMM approximates with the free-space Green's functions.
//   (A u)_ijk = (6 u_ijk - u_{i+-1,j,k} - u_{i,j+-1,k} - u_{i,j,k+-1}) / h^2 - shift u_ijk,
// shift = 0 (Laplace) or kappa^2 (Helmholtz), u = 0 outside the m x m x m
// interior grid, index (k m + j) m + i.
#include <cmath>

#include "plan.cuh"

namespace fmm {

namespace {

__global__ void k_laplace7(const double *__restrict__ u, double *__restrict__ out, int64_t m,
                           double inv_h2, double shift) {
  const int64_t total = m * m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % m, j = (t / m) % m, k = t / (m * m);
    double s = 6.0 * u[t];
    if (i > 0) s -= u[t - 1];
    if (i + 1 < m) s -= u[t + 1];
    if (j > 0) s -= u[t - m];
    if (j + 1 < m) s -= u[t + m];
    if (k > 0) s -= u[t - m * m];
    if (k + 1 < m) s -= u[t + m * m];
    out[t] = s * inv_h2 - shift * u[t];
  }
}

}  // namespace

}  // namespace fmm

using namespace fmm;

static fmm_status apply7(const double *d_u, double *d_out, int64_t m, double h, double shift,
                         void *stream, const char *name) {
  if (m < 0 || !(h > 0.0) || !std::isfinite(shift))
    return record_error(FMM_ERR_INVALID_ARG, std::string(name) + ": m < 0, h <= 0 or bad shift");
  if (m > 0 && (!d_u || !d_out))
    return record_error(FMM_ERR_INVALID_ARG, std::string(name) + ": NULL grid pointer");
  if (m > 2097151) return record_error(FMM_ERR_INVALID_ARG, std::string(name) + ": m too large");
  if (m == 0) return FMM_OK;
  try {
    const int64_t total = m * m * m;
    const int blocks = (int)std::min<int64_t>(ceil_div(total, (int64_t)256), 152 * 16);
    k_laplace7<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_u, d_out, m, 1.0 / (h * h), shift);
    FMM_LAUNCH_CHECK();
    return FMM_OK;
  } catch (const Error &e) {
    return record_error(e.status, e.what());
  }
}

extern "C" fmm_status fmm_laplace7_apply(const double *d_u, double *d_out, int64_t m, double h,
                                         void *stream) {
  return apply7(d_u, d_out, m, h, 0.0, stream, "fmm_laplace7_apply");
}

extern "C" fmm_status fmm_helmholtz7_apply(const double *d_u, double *d_out, int64_t m, double h,
                                           double kappa, void *stream) {
  if (!std::isfinite(kappa))
    return record_error(FMM_ERR_INVALID_ARG, "fmm_helmholtz7_apply: kappa not finite");
  return apply7(d_u, d_out, m, h, kappa * kappa, stream, "fmm_helmholtz7_apply");
}

// lbo_evolve_homogeneous: explicit time integration of the spatially
// homogeneous equations of Sec. 4.2,
//     df/dt = Q(f, f)      (LBO_EVOLVE_QUADRATIC)
//     df/dt = L_M[f]       (LBO_EVOLVE_LINEARIZED; M of the given params),
// with the classical fourth-order Runge-Kutta scheme (the paper's time
// discretisation, step 0.1):
//     k1 = F(f), k2 = F(f + dt/2 k1), k3 = F(f + dt/2 k2), k4 = F(f + dt k3),
//     f <- f + dt/6 (k1 + 2 k2 + 2 k3 + k4),
// every operator evaluation through the plan (its precision, kernel set and
// fixes apply at each evaluation: the mass fix of Sec. 4.2 per step).  The
// linearized form applies L to f itself (L[M] = 0, so L[f] = L[f - M]) and
// uses the Maxwellian cache for all its steps.
#include <cuda_runtime.h>

#include <algorithm>

#include "lbo_internal.h"

namespace lbo {
namespace {

// y = a + s b
__global__ void k_combine2(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                           double s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a[i] + s * b[i];
}

// acc = c k (first) or acc + c k
__global__ void k_accumulate(double* __restrict__ acc, const double* __restrict__ k, double c, int first, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc[i] = first ? c * k[i] : acc[i] + c * k[i];
}

// f = f + s (acc + k)
__global__ void k_rk4_finish(double* __restrict__ f, const double* __restrict__ acc, const double* __restrict__ k,
                             double s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    f[i] += s * (acc[i] + k[i]);
}

}  // namespace
}  // namespace lbo

using namespace lbo;

extern "C" lbo_status lbo_evolve_homogeneous(lbo_plan* p, int mode, const double* params, double* f, int batch,
                                             double dt, int nsteps) {
  if (!p || !f || batch < 0 || nsteps < 0 || !(dt > 0.0)) return LBO_EINVAL;
  if (mode != LBO_EVOLVE_QUADRATIC && mode != LBO_EVOLVE_LINEARIZED) return LBO_EINVAL;
  if (mode == LBO_EVOLVE_LINEARIZED && !params) return LBO_EINVAL;
  if (batch == 0 || nsteps == 0) return LBO_OK;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, f) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error_text("evolve: f must be a device pointer");
    return LBO_EINVAL;
  }
  const size_t n = (size_t)batch * p->N * p->N * p->N;
  double* buf = nullptr;  // y, k, acc
  cudaError_t e = cudaMalloc(&buf, 3 * n * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error_text("evolve: stage buffers");
    return LBO_ENOMEM;
  }
  double *y = buf, *k = buf + n, *acc = buf + 2 * n;
  cudaStream_t s = p->stream;
  const int grid = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  // the linearized form keeps the Maxwellian factors cached for every step
  // (unless the caller already cached them for these params)
  bool own_cache = false;
  lbo_status st = LBO_OK;
  if (mode == LBO_EVOLVE_LINEARIZED && !(p->mc_valid && p->mc_params == params && p->mc_batch == batch)) {
    st = lbo_plan_cache_maxwellians(p, params, batch);
    own_cache = st == LBO_OK;
  }
  auto F = [&](const double* x, double* out) -> lbo_status {
    return mode == LBO_EVOLVE_LINEARIZED ? lbo_apply_linearized(p, params, x, out, batch)
                                         : lbo_apply_quadratic(p, x, out, batch);
  };
  int launches = 0;
  for (int it = 0; it < nsteps && st == LBO_OK; ++it) {
    st = F(f, k);  // k1
    if (st != LBO_OK) break;
    launches += p->last_launches;
    LBO_LAUNCH(p, "rk4_accumulate", s, k_accumulate, grid, 256, 0, acc, k, 1.0, 1, n);
    LBO_LAUNCH(p, "rk4_stage", s, k_combine2, grid, 256, 0, y, f, k, 0.5 * dt, n);
    for (int stage = 2; stage <= 3 && st == LBO_OK; ++stage) {  // k2, k3
      st = F(y, k);
      launches += p->last_launches;
      LBO_LAUNCH(p, "rk4_accumulate", s, k_accumulate, grid, 256, 0, acc, k, 2.0, 0, n);
      LBO_LAUNCH(p, "rk4_stage", s, k_combine2, grid, 256, 0, y, f, k, stage == 2 ? 0.5 * dt : dt, n);
    }
    if (st != LBO_OK) break;
    st = F(y, k);  // k4
    launches += p->last_launches;
    LBO_LAUNCH(p, "rk4_finish", s, k_rk4_finish, grid, 256, 0, f, acc, k, dt / 6.0, n);
    launches += 6;
  }
  if (own_cache) lbo_plan_cache_maxwellians(p, nullptr, 0);
  e = cudaStreamSynchronize(s);  // before the stage buffers are freed
  cudaFree(buf);
  p->last_launches = launches;
  if (st != LBO_OK) return st;
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "evolve");
}

// Primitives on one block of cells of the 1-D slab (Sec. 5 and the
// supplement's fully discrete scheme) for a solver whose cells are split
// over several GPUs: each GPU owns a contiguous block [c0, c0 + nx) and the
// cells next to it (a neighbour block's boundary cell, or a wall's ghost
// cell) are given explicitly.  A host-side driver composes these into the
// modified Newton / flexible GMRES iteration, exchanging the boundary cells
// between neighbours and summing dot products, norms and masses over the
// GPUs (paper_2503_09580_gb300/distributed.py).  Layout: cells one after the
// other, each N^3 doubles in the library's centred order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "lbo_internal.h"

namespace lbo {
namespace {

constexpr int kBlocks = 304, kThreads = 256;

int grid_of(size_t len) { return (int)std::min<size_t>((len + 255) / 256, 152 * 8); }

// out_j = v1^+ (v_j - v_{j-1}) / dx + v1^- (v_{j+1} - v_j) / dx, with v_{-1} =
// gl and v_{nx} = gr (0 where null)
__global__ void k_block_transport(const double* __restrict__ v, const double* __restrict__ gl,
                                  const double* __restrict__ gr, double* __restrict__ out, int N, int nx, double h,
                                  double dx) {
  const size_t n3 = (size_t)N * N * N, len = n3 * nx;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / n3);
    const size_t k = t % n3;
    const double v1 = (int(k / ((size_t)N * N)) - N / 2) * h;
    const double c = v[t];
    if (v1 > 0) {
      const double left = j == 0 ? (gl ? gl[k] : 0.0) : v[t - n3];
      out[t] = v1 * (c - left) / dx;
    } else {
      const double right = j == nx - 1 ? (gr ? gr[k] : 0.0) : v[t + n3];
      out[t] = v1 * (right - c) / dx;
    }
  }
}

// (v1^+ D^- + v1^- D^+ + nu_j/Kn + shift) z = r on the block, the incoming
// values z_{-1} = il (for v1 > 0) and z_{nx} = ir (for v1 < 0) given (0 where
// null).  direction: +1 only the velocities with v1 > 0, -1 only v1 < 0,
// 0 all (v1 = 0 is solved with the v1 > 0 half).
__global__ void k_block_sweep(const double* __restrict__ r, const double* __restrict__ nu,
                              const double* __restrict__ il, const double* __restrict__ ir, double* __restrict__ z,
                              int N, int nx, double h, double dx, double kn, double shift, int direction) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n3; k += (size_t)gridDim.x * blockDim.x) {
    const double v1 = (int(k / ((size_t)N * N)) - N / 2) * h;
    const double c = fabs(v1) / dx;
    if (v1 > 0) {
      if (direction < 0) continue;
      double prev = il ? il[k] : 0.0;
      for (int j = 0; j < nx; ++j) {
        prev = (r[(size_t)j * n3 + k] + c * prev) / (c + nu[j] / kn + shift);
        z[(size_t)j * n3 + k] = prev;
      }
    } else if (v1 < 0) {
      if (direction > 0) continue;
      double prev = ir ? ir[k] : 0.0;
      for (int j = nx - 1; j >= 0; --j) {
        prev = (r[(size_t)j * n3 + k] + c * prev) / (c + nu[j] / kn + shift);
        z[(size_t)j * n3 + k] = prev;
      }
    } else {
      if (direction < 0) continue;
      for (int j = 0; j < nx; ++j) z[(size_t)j * n3 + k] = r[(size_t)j * n3 + k] / (nu[j] / kn + shift);
    }
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// part[b K + k] = block b's share of <V_k, y>
__global__ void __launch_bounds__(kThreads) k_vdots(const double* __restrict__ V, size_t ld, int K,
                                                    const double* __restrict__ y, size_t len,
                                                    double* __restrict__ part) {
  __shared__ double sh[32];
  for (int k = 0; k < K; ++k) {
    double a = 0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
      a += V[(size_t)k * ld + e] * y[e];
    const double s = block_sum(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x * K + k] = s;
  }
}

// out[k] = sum over the blocks in a fixed order (deterministic)
__global__ void k_vdots_finish(const double* __restrict__ part, int nb, int K, double* __restrict__ out) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b * K + k];
    out[k] = s;
  }
}

__global__ void k_vaxpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, size_t len) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + b * y[e];
}

// y -= sum_k c[k] V_k
__global__ void k_vcomb(double* __restrict__ y, const double* __restrict__ V, size_t ld, int K,
                        const double* __restrict__ c, size_t len) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int k = 0; k < K; ++k) s += c[k] * V[(size_t)k * ld + e];
    y[e] -= s;
  }
}

// per-cell moments (Sec. 2.1): params[j] = (rho, u1, u2, u3, theta), nu[j] = rho
__global__ void __launch_bounds__(kThreads) k_block_moments(const double* __restrict__ f, int N, double h,
                                                            double* __restrict__ params, double* __restrict__ nu) {
  __shared__ double sh[32];
  const size_t n3 = (size_t)N * N * N;
  const double* x = f + (size_t)blockIdx.x * n3;
  double m[5] = {0, 0, 0, 0, 0};
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    const int i3 = (int)(t % N), i2 = (int)((t / N) % N), i1 = (int)(t / ((size_t)N * N));
    const double v1 = (i1 - N / 2) * h, v2 = (i2 - N / 2) * h, v3 = (i3 - N / 2) * h, y = x[t];
    m[0] += y;
    m[1] += v1 * y;
    m[2] += v2 * y;
    m[3] += v3 * y;
    m[4] += (v1 * v1 + v2 * v2 + v3 * v3) * y;
  }
  double s[5];
  for (int a = 0; a < 5; ++a) s[a] = block_sum(m[a], sh);
  if (threadIdx.x == 0) {
    const double h3 = h * h * h, rho = h3 * s[0];
    const double u1 = h3 * s[1] / rho, u2 = h3 * s[2] / rho, u3 = h3 * s[3] / rho;
    const double e = h3 * s[4] - rho * (u1 * u1 + u2 * u2 + u3 * u3);
    double* p = params + 5 * blockIdx.x;
    p[0] = rho;
    p[1] = u1;
    p[2] = u2;
    p[3] = u3;
    p[4] = e / (3.0 * rho);
    if (nu) nu[blockIdx.x] = rho;
  }
}

// part[b] = block b's share of h^3 sum v1^- x (side 0) or h^3 sum v1^+ x (side 1)
__global__ void __launch_bounds__(kThreads) k_cell_flux(const double* __restrict__ x, int N, double h, int side,
                                                        double* __restrict__ part) {
  __shared__ double sh[32];
  const size_t n3 = (size_t)N * N * N;
  double a = 0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n3; t += (size_t)gridDim.x * blockDim.x) {
    const double v1 = (int(t / ((size_t)N * N)) - N / 2) * h;
    a += (side == 0 ? fmin(v1, 0.0) : fmax(v1, 0.0)) * x[t];
  }
  const double s = block_sum(a, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = h * h * h * s;
}

// out = scale (2 pi theta)^{-3/2} exp(-|v - u|^2 / (2 theta))
__global__ void k_maxwellian_cell(double* __restrict__ out, int N, double h, double theta, double u1, double u2,
                                  double u3, double scale) {
  const size_t n3 = (size_t)N * N * N;
  const double pref = scale * pow(2.0 * 3.141592653589793 * theta, -1.5);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n3; t += (size_t)gridDim.x * blockDim.x) {
    const int i3 = (int)(t % N), i2 = (int)((t / N) % N), i1 = (int)(t / ((size_t)N * N));
    const double d1 = (i1 - N / 2) * h - u1, d2 = (i2 - N / 2) * h - u2, d3 = (i3 - N / 2) * h - u3;
    out[t] = pref * exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * theta));
  }
}

// device scratch of the plan for the reductions (grown on demand; freed
// with the plan)
lbo_status reduce_scratch(lbo_plan* p, int K, double** part, double** out) {
  const size_t need = (size_t)kBlocks * K + K;
  if (need > p->blk_red_cap) {
    if (p->blk_red) cudaFree(p->blk_red);
    p->blk_red = nullptr;
    p->blk_red_cap = 0;
    if (cudaMalloc(&p->blk_red, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      set_error_text("slab block: reduction scratch");
      return LBO_ENOMEM;
    }
    p->blk_red_cap = need;
  }
  *part = p->blk_red;
  *out = p->blk_red + (size_t)kBlocks * K;
  return LBO_OK;
}

double slab_h(const lbo_plan* p) { return 2.0 * p->L / p->N; }

}  // namespace
}  // namespace lbo

using namespace lbo;

extern "C" {

lbo_status lbo_slab_block_transport(lbo_plan* p, const double* v, const double* ghost_left, const double* ghost_right,
                                    double* out, int nx, double dx) {
  if (!p || !v || !out || nx < 1 || !(dx > 0)) return LBO_EINVAL;
  const size_t len = (size_t)nx * p->N * p->N * p->N;
  LBO_LAUNCH(p, "block_transport", p->stream, k_block_transport, grid_of(len), kThreads, 0, v, ghost_left,
             ghost_right, out, p->N, nx, slab_h(p), dx);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "block transport");
}

lbo_status lbo_slab_block_sweep(lbo_plan* p, const double* r, const double* nu, const double* in_left,
                                const double* in_right, double* z, int nx, double dx, double kn, double shift,
                                int direction) {
  if (!p || !r || !nu || !z || nx < 1 || !(dx > 0) || !(kn > 0) || direction < -1 || direction > 1)
    return LBO_EINVAL;
  const size_t n3 = (size_t)p->N * p->N * p->N;
  LBO_LAUNCH(p, "block_sweep", p->stream, k_block_sweep, grid_of(n3), kThreads, 0, r, nu, in_left, in_right, z,
             p->N, nx, slab_h(p), dx, kn, shift, direction);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "block sweep");
}

lbo_status lbo_slab_block_moments(lbo_plan* p, const double* f, int nx, double* params, double* nu) {
  if (!p || !f || !params || nx < 1) return LBO_EINVAL;
  LBO_LAUNCH(p, "block_moments", p->stream, k_block_moments, nx, kThreads, 0, f, p->N, slab_h(p), params, nu);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "block moments");
}

lbo_status lbo_slab_cell_flux(lbo_plan* p, const double* cell, int side, double* host_out) {
  if (!p || !cell || !host_out || (side != 0 && side != 1)) return LBO_EINVAL;
  double *part, *out;
  lbo_status st = reduce_scratch(p, 1, &part, &out);
  if (st != LBO_OK) return st;
  const size_t n3 = (size_t)p->N * p->N * p->N;
  LBO_LAUNCH(p, "cell_flux", p->stream, k_cell_flux, kBlocks, kThreads, 0, cell, p->N, slab_h(p), side, part);
  LBO_LAUNCH(p, "cell_flux_finish", p->stream, k_vdots_finish, 1, 32, 0, part, kBlocks, 1, out);
  cudaError_t e = cudaMemcpyAsync(host_out, out, sizeof(double), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  (void)n3;
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "cell flux");
}

lbo_status lbo_slab_maxwellian_cell(lbo_plan* p, double theta, const double* u, double scale, double* out) {
  if (!p || !u || !out || !(theta > 0)) return LBO_EINVAL;
  const size_t n3 = (size_t)p->N * p->N * p->N;
  LBO_LAUNCH(p, "maxwellian_cell", p->stream, k_maxwellian_cell, grid_of(n3), kThreads, 0, out, p->N, slab_h(p),
             theta, u[0], u[1], u[2], scale);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "maxwellian cell");
}

lbo_status lbo_vec_dots(lbo_plan* p, const double* V, size_t ld, int K, const double* y, size_t len,
                        double* host_out) {
  if (!p || !V || !y || !host_out || K < 1 || K > 512) return LBO_EINVAL;
  double *part, *out;
  lbo_status st = reduce_scratch(p, K, &part, &out);
  if (st != LBO_OK) return st;
  LBO_LAUNCH(p, "vec_dots", p->stream, k_vdots, kBlocks, kThreads, 0, V, ld, K, y, len, part);
  LBO_LAUNCH(p, "vec_dots_finish", p->stream, k_vdots_finish, 1, 256, 0, part, kBlocks, K, out);
  cudaError_t e = cudaMemcpyAsync(host_out, out, sizeof(double) * K, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "vec dots");
}

lbo_status lbo_vec_axpby(lbo_plan* p, double* y, const double* x, double a, double b, size_t len) {
  if (!p || !y || !x) return LBO_EINVAL;
  LBO_LAUNCH(p, "vec_axpby", p->stream, k_vaxpby, grid_of(len), kThreads, 0, y, x, a, b, len);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "vec axpby");
}

lbo_status lbo_vec_combination(lbo_plan* p, double* y, const double* V, size_t ld, int K, const double* c_host,
                               size_t len) {
  if (!p || !y || !V || !c_host || K < 1 || K > 512) return LBO_EINVAL;
  double *part, *out;
  lbo_status st = reduce_scratch(p, K, &part, &out);
  if (st != LBO_OK) return st;
  cudaError_t e = cudaMemcpyAsync(out, c_host, sizeof(double) * K, cudaMemcpyHostToDevice, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "vec combination");
  LBO_LAUNCH(p, "vec_combination", p->stream, k_vcomb, grid_of(len), kThreads, 0, y, V, ld, K, out, len);
  e = cudaStreamSynchronize(p->stream);  // c_host may be reused by the caller at once
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "vec combination");
}

}  // extern "C"

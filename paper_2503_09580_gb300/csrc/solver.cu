// Modified Newton / flexible GMRES solver (Sec. 5 and the supplement's fully
// discrete scheme) on top of a plan's L[g] and Q(f,f).  Host-side Arnoldi on
// small matrices; every long-vector operation is an FP64 kernel here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lbo_internal.h"

namespace lbo {
namespace {

constexpr int RED_BLOCKS = 304;  // 2 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int DOT_TILE = 8;

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
  return t;  // valid in thread 0
}

// part[b*K + k] = sum over this block's elements of V_k[e] * y[e], k < K
__global__ void __launch_bounds__(RED_THREADS) k_dots(const double* __restrict__ V, size_t ld, int K,
                                                      const double* __restrict__ y, size_t len,
                                                      double* __restrict__ part) {
  __shared__ double sh[32];
  for (int k0 = 0; k0 < K; k0 += DOT_TILE) {
    double acc[DOT_TILE];
#pragma unroll
    for (int t = 0; t < DOT_TILE; ++t) acc[t] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
      const double ye = y[e];
#pragma unroll
      for (int t = 0; t < DOT_TILE; ++t)
        if (k0 + t < K) acc[t] += V[(size_t)(k0 + t) * ld + e] * ye;
    }
#pragma unroll
    for (int t = 0; t < DOT_TILE; ++t) {
      double s = block_sum(acc[t], sh);
      if (threadIdx.x == 0 && k0 + t < K) part[blockIdx.x * K + k0 + t] = s;
    }
  }
}

// out[k] = sum_b part[b*K + k] (fixed order: deterministic)
__global__ void k_reduce_parts(const double* __restrict__ part, int nb, int K, double* __restrict__ out) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b * K + k];
    out[k] = s;
  }
}

// y -= sum_k c[k] V_k
__global__ void k_sub_combination(double* __restrict__ y, const double* __restrict__ V, size_t ld, int K,
                                  const double* __restrict__ c, size_t len) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int k = 0; k < K; ++k) s += c[k] * V[(size_t)k * ld + e];
    y[e] -= s;
  }
}

// y = a x + b y  (a, b on the host)
__global__ void k_scale(double* y, double a, size_t len) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    y[e] *= a;
}

__global__ void k_axpby(double* __restrict__ y, const double* __restrict__ x, double a, double b, size_t len) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    y[e] = a * x[e] + b * y[e];
}

// local Maxwellian parameters of each cell: rho, u, theta (Sec. 2.1), FP64
__global__ void __launch_bounds__(512) k_cell_moments(const double* __restrict__ f, double* __restrict__ params,
                                                     double* __restrict__ nu, int N, double h) {
  __shared__ double sh[32];
  __shared__ double mom[4];
  const size_t n3 = (size_t)N * N * N;
  const double* x = f + blockIdx.x * n3;
  double m0 = 0, m1 = 0, m2 = 0, m3 = 0;
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    const int i3 = (int)(t % N), i2 = (int)((t / N) % N), i1 = (int)(t / ((size_t)N * N));
    const double y = x[t];
    m0 += y;
    m1 += (i1 - N / 2) * h * y;
    m2 += (i2 - N / 2) * h * y;
    m3 += (i3 - N / 2) * h * y;
  }
  double r0 = block_sum(m0, sh);
  if (threadIdx.x == 0) mom[0] = r0;
  double r1 = block_sum(m1, sh);
  if (threadIdx.x == 0) mom[1] = r1;
  double r2 = block_sum(m2, sh);
  if (threadIdx.x == 0) mom[2] = r2;
  double r3 = block_sum(m3, sh);
  if (threadIdx.x == 0) mom[3] = r3;
  __syncthreads();
  const double h3 = h * h * h, rho = h3 * mom[0];
  const double u1 = h3 * mom[1] / rho, u2 = h3 * mom[2] / rho, u3 = h3 * mom[3] / rho;
  double e = 0;
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    const int i3 = (int)(t % N), i2 = (int)((t / N) % N), i1 = (int)(t / ((size_t)N * N));
    const double c1 = (i1 - N / 2) * h - u1, c2 = (i2 - N / 2) * h - u2, c3 = (i3 - N / 2) * h - u3;
    e += (c1 * c1 + c2 * c2 + c3 * c3) * x[t];
  }
  double re = block_sum(e, sh);
  if (threadIdx.x == 0) {
    double* p = params + 5 * blockIdx.x;
    p[0] = rho;
    p[1] = u1;
    p[2] = u2;
    p[3] = u3;
    p[4] = h3 * re / (3.0 * rho);
    if (nu) nu[blockIdx.x] = rho;
  }
}

// res[0] = -kL h^3 sum v1^- v_1, res[1] = kR h^3 sum v1^+ v_nx (wall densities),
// res[2] = dx h^3 sum v (total mass); blocks 0, 1 the walls, the rest the mass
__global__ void __launch_bounds__(RED_THREADS) k_wall_mass(const double* __restrict__ v, int N, int nx, double h,
                                                           double dx, double kL, double kR,
                                                           double* __restrict__ part, double* __restrict__ res) {
  __shared__ double sh[32];
  const size_t n3 = (size_t)N * N * N, len = n3 * nx;
  const double h3 = h * h * h;
  if (blockIdx.x < 2) {
    const double* x = v + (blockIdx.x == 0 ? 0 : (size_t)(nx - 1) * n3);
    double a = 0;
    for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
      const double v1 = (int(t / ((size_t)N * N)) - N / 2) * h;
      a += (blockIdx.x == 0 ? fmin(v1, 0.0) : fmax(v1, 0.0)) * x[t];
    }
    double s = block_sum(a, sh);
    if (threadIdx.x == 0) res[blockIdx.x] = blockIdx.x == 0 ? -kL * h3 * s : kR * h3 * s;
  } else {
    double a = 0;
    const int nb = gridDim.x - 2, b = blockIdx.x - 2;
    for (size_t e = b * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)nb * blockDim.x) a += v[e];
    double s = block_sum(a, sh);
    if (threadIdx.x == 0) part[b] = s;
  }
}

__global__ void k_mass_finish(const double* __restrict__ part, int nb, double w, double* __restrict__ res) {
  if (threadIdx.x == 0) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b];
    res[2] = w * s;
  }
}

// out = T v * cT + y * cY + e * m(v) * cE, T the upwind transport with
// diffuse-wall ghost cells (densities res[0], res[1]), m(v) = res[2].
// Inflow sides pass a fixed ghost factor gL / gR >= 0 (1 for the residual,
// 0 for the Newton correction); walls pass -1 and use res[0], res[1].
__global__ void k_transport(const double* __restrict__ v, const double* __restrict__ y,
                            const double* __restrict__ e, const double* __restrict__ res,
                            const double* __restrict__ WL, const double* __restrict__ WR,
                            double* __restrict__ out, int N, int nx, double h, double dx, double cT, double cY,
                            double cE, double gL, double gR, double cV) {
  const size_t n3 = (size_t)N * N * N, len = n3 * nx;
  const double sL = gL >= 0 ? gL : res[0], sR = gR >= 0 ? gR : res[1], mv = res[2];
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / n3);
    const size_t k = t % n3;
    const double v1 = (int(k / ((size_t)N * N)) - N / 2) * h;
    const double c = v[t];
    double tv;
    if (v1 > 0) {
      const double left = j == 0 ? sL * WL[k] : v[t - n3];
      tv = v1 * (c - left) / dx;
    } else {
      const double right = j == nx - 1 ? sR * WR[k] : v[t + n3];
      tv = v1 * (right - c) / dx;
    }
    double o = cT * tv + cV * c;
    if (y) o += cY * y[t];
    if (e) o += cE * mv * e[t];
    out[t] = o;
  }
}

// Upwind sweep of the source iteration (Eq. (5.7)):
// (v1^+ D^- + v1^- D^+ + nu_j/Kn) z = r, ghost values of z taken as 0.
__global__ void k_sweep(const double* __restrict__ r, double* __restrict__ z, const double* __restrict__ nu, int N,
                        int nx, double h, double dx, double kn, double sh) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n3; k += (size_t)gridDim.x * blockDim.x) {
    const double v1 = (int(k / ((size_t)N * N)) - N / 2) * h;
    const double c = fabs(v1) / dx;
    if (v1 > 0) {
      double prev = 0;
      for (int j = 0; j < nx; ++j) {
        prev = (r[(size_t)j * n3 + k] + c * prev) / (c + nu[j] / kn + sh);
        z[(size_t)j * n3 + k] = prev;
      }
    } else if (v1 < 0) {
      double prev = 0;
      for (int j = nx - 1; j >= 0; --j) {
        prev = (r[(size_t)j * n3 + k] + c * prev) / (c + nu[j] / kn + sh);
        z[(size_t)j * n3 + k] = prev;
      }
    } else {
      for (int j = 0; j < nx; ++j) z[(size_t)j * n3 + k] = r[(size_t)j * n3 + k] / (nu[j] / kn + sh);
    }
  }
}

int grid_for(size_t len) {
  size_t b = (len + 255) / 256;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

// Euclidean dot products res[k] = <V_k, y>, k < K; result copied to host.
lbo_status dots(lbo_solver* S, const double* Vb, size_t ld, int K, const double* y, double* host_out) {
  cudaStream_t s = S->plan->stream;
  LBO_LAUNCH(S->plan, "solver_dots", s, k_dots, RED_BLOCKS, RED_THREADS, 0, Vb, ld, K, y, S->len, S->part);
  LBO_LAUNCH(S->plan, "solver_reduce", s, k_reduce_parts, 1, 256, 0, S->part, RED_BLOCKS, K, S->res + 8);
  cudaError_t e = cudaMemcpyAsync(host_out, S->res + 8, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "solver dots");
}

double norm2(lbo_solver* S, const double* y, lbo_status* st) {
  double v = 0;
  *st = dots(S, y, 0, 1, y, &v);
  return std::sqrt(v);
}

// wall densities and total mass of v into S->res[0..2]
void wall_mass(lbo_solver* S, const double* v) {
  cudaStream_t s = S->plan->stream;
  const int nb = RED_BLOCKS;
  LBO_LAUNCH(S->plan, "solver_wall_mass", s, k_wall_mass, nb + 2, RED_THREADS, 0, v, S->N, S->nx, S->h, S->dx,
             S->kL, S->kR, S->part, S->res);
  LBO_LAUNCH(S->plan, "solver_mass_finish", s, k_mass_finish, 1, 32, 0, S->part, nb, S->dx * S->h * S->h * S->h,
             S->res);
}

bool bordered(const lbo_solver* S) {
  return S->pb.kind == LBO_PROBLEM_SLAB && S->pb.bc_left == LBO_BC_WALL && S->pb.bc_right == LBO_BC_WALL;
}

// Lv = J_Q v = (Q(f + s v) - Q(f - s v)) / (2 s), s = |f| / |v|: exact for
// the bilinear Q up to rounding, balanced so that s v is of the size of f.
lbo_status exact_jacobian_q(lbo_solver* S, const double* v) {
  cudaStream_t s = S->plan->stream;
  lbo_status st = LBO_OK;
  const double vn = norm2(S, v, &st);
  if (st != LBO_OK) return st;
  if (!(vn > 0)) {
    cudaMemsetAsync(S->Lv, 0, sizeof(double) * S->len, s);
    return LBO_OK;
  }
  const double sc = S->fnorm > 0 ? S->fnorm / vn : 1.0;
  for (int side = 0; side < 2; ++side) {
    double* x = side == 0 ? S->ja : S->jb;
    cudaMemcpyAsync(x, S->fcur, sizeof(double) * S->len, cudaMemcpyDeviceToDevice, s);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, x, v, side == 0 ? sc : -sc, 1.0,
               S->len);
  }
  S->plan->stream = s;
  st = lbo_apply_quadratic(S->plan, S->ja, S->Lv, S->nx);  // Q(f + s v)
  if (st == LBO_OK) st = lbo_apply_quadratic(S->plan, S->jb, S->ja, S->nx);  // Q(f - s v)
  if (st != LBO_OK) return st;
  LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, S->Lv, S->ja, -0.5 / sc, 0.5 / sc,
             S->len);
  return LBO_OK;
}

// out = A' v:  SLAB: T v - L v / Kn + e m(v) + v / dtau;  HOMOGENEOUS: v - dt L v
// (L v replaced by the exact J_Q v when the problem asks for the exact Jacobian)
// collisions = false drops the collision term (SLAB only): the transport,
// border and shift parts alone, for the transport-only coarse operator
lbo_status apply_op(lbo_solver* S, const double* v, double* out, bool border = true, bool collisions = true) {
  if (S->mixed) return collisions ? mixed_apply_op(S, v, out) : LBO_EUNSUPPORTED;
  if (!collisions && S->pb.kind != LBO_PROBLEM_SLAB) return LBO_EINVAL;
  lbo_status st = !collisions          ? LBO_OK
                  : S->pb.jacobian == 1 ? exact_jacobian_q(S, v)
                                        : lbo_apply_linearized(S->plan, S->params, v, S->Lv, S->nx);
  if (st != LBO_OK) return st;
  cudaStream_t s = S->plan->stream;
  if (S->pb.kind == LBO_PROBLEM_SLAB) {
    wall_mass(S, v);
    // the mass border e m(v) only where both sides are walls: an inflow side
    // fixes the incoming ghost values, so the operator has no mass null mode
    const double* ev = border && bordered(S) ? S->evec : nullptr;
    const double* lv = collisions ? S->Lv : nullptr;
    LBO_LAUNCH(S->plan, "solver_transport", s, k_transport, grid_for(S->len), 256, 0, v, lv, ev, S->res,
               S->WL, S->WR, out, S->N, S->nx, S->h, S->dx, 1.0, -1.0 / S->pb.kn, 1.0,
               S->pb.bc_left == LBO_BC_INFLOW ? 0.0 : -1.0, S->pb.bc_right == LBO_BC_INFLOW ? 0.0 : -1.0, S->shift);
  } else {
    if (out != v) cudaMemcpyAsync(out, v, sizeof(double) * S->len, cudaMemcpyDeviceToDevice, s);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, out, S->Lv, -S->pb.dt, 1.0, S->len);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "solver operator");
}

lbo_status apply_precond(lbo_solver* S, const double* v, double* z);

lbo_status sweep_only(lbo_solver* S, const double* v, double* z) {
  LBO_LAUNCH(S->plan, "solver_sweep", S->plan->stream, k_sweep, grid_for(S->n3), 256, 0, v, z, S->nu, S->N, S->nx,
             S->h, S->dx, S->pb.kn, S->shift);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "sweep");
}

// Nonlinear residual into out (and its weighted norm).
lbo_status residual(lbo_solver* S, const double* f, const double* f_prev, double* out, double* nrm) {
  if (S->mixed) return mixed_residual(S, f, out, nrm);
  lbo_plan* qp = S->rplan ? S->rplan : S->plan;
  qp->stream = S->plan->stream;
  lbo_status st = lbo_apply_quadratic(qp, f, S->Qf, S->nx);
  if (st != LBO_OK) return st;
  cudaStream_t s = S->plan->stream;
  if (S->pb.kind == LBO_PROBLEM_SLAB) {
    wall_mass(S, f);
    LBO_LAUNCH(S->plan, "solver_transport", s, k_transport, grid_for(S->len), 256, 0, f, S->Qf, (const double*)nullptr,
               S->res, S->WL, S->WR, out, S->N, S->nx, S->h, S->dx, 1.0, -1.0 / S->pb.kn, 0.0,
               S->pb.bc_left == LBO_BC_INFLOW ? 1.0 : -1.0, S->pb.bc_right == LBO_BC_INFLOW ? 1.0 : -1.0, 0.0);
  } else {
    // F = f - f_prev - dt Q
    cudaMemcpyAsync(out, f, sizeof(double) * S->len, cudaMemcpyDeviceToDevice, s);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, out, f_prev, -1.0, 1.0, S->len);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, out, S->Qf, -S->pb.dt, 1.0, S->len);
  }
  if (nrm) {
    double v = norm2(S, out, &st);
    if (st != LBO_OK) return st;
    *nrm = v * std::sqrt(S->wnorm);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "solver residual");
}

// Restarted flexible GMRES on A' x = rhs, x0 = 0 (right preconditioning).
lbo_status fgmres(lbo_solver* S, lbo_newton_stats* ns) {
  const int m = S->m;
  const size_t len = S->len;
  cudaStream_t s = S->plan->stream;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gam(m + 1), y(m), hv(m + 1), hv2(m + 1);
  lbo_status st;
  cudaMemsetAsync(S->x, 0, sizeof(double) * len, s);
  double rhs_norm = norm2(S, S->rhs, &st);
  if (st != LBO_OK) return st;
  ns->rhs_norm = rhs_norm * std::sqrt(S->wnorm);
  const double tol = std::fmax(S->pb.krylov_rtol * rhs_norm, S->pb.krylov_atol / std::sqrt(S->wnorm));
  ns->krylov_iterations = 0;
  ns->restarts = 0;
  ns->status = LBO_OK;
  if (rhs_norm == 0.0) return LBO_OK;
  if (!std::isfinite(rhs_norm)) {
    ns->status = LBO_ENAN;
    return LBO_ENAN;
  }
  // r0 = rhs
  cudaMemcpyAsync(S->V, S->rhs, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
  double beta = rhs_norm;
  bool done = false;
  // the learned preconditioner gets half the iteration budget; if it has not
  // converged by then, the solve continues from the current iterate with the
  // plain sweep (the exact operator still measures convergence)
  S->force_sweep = false;
  const bool learned = S->pb.precond == LBO_PRECOND_LEARNED;
  const int learned_budget = S->pb.krylov_maxit / 2;
  while (!done) {
    LBO_LAUNCH(S->plan, "solver_scale", s, k_scale, grid_for(len), 256, 0, S->V, 1.0 / beta, len);
    std::fill(gam.begin(), gam.end(), 0.0);
    gam[0] = beta;
    int k = 0;
    for (; k < m; ++k) {
      double* vk = S->V + (size_t)k * len;
      double* zk = S->Z + (size_t)k * len;
      st = apply_precond(S, vk, zk);
      if (st != LBO_OK) return st;
      st = apply_op(S, zk, S->w);
      if (st != LBO_OK) return st;
      if (S->pb.kind == LBO_PROBLEM_SLAB) {
        // training pair (A z_k, z_k) for the learned preconditioner, if collecting
        st = network_record(S, S->w, zk, S->Lv, sweep_only);
        if (st != LBO_OK) return st;
      }
      // classical Gram-Schmidt, two passes, FP64
      for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        st = dots(S, S->V, len, k + 1, S->w, hv.data());
        if (st != LBO_OK) return st;
        cudaMemcpyAsync(S->res + 8, hv.data(), sizeof(double) * (k + 1), cudaMemcpyHostToDevice, s);
        LBO_LAUNCH(S->plan, "solver_sub", s, k_sub_combination, grid_for(len), 256, 0, S->w, S->V, len, k + 1,
                   S->res + 8, len);
        for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] += hv[i];
      }
      double hn = norm2(S, S->w, &st);
      if (st != LBO_OK) return st;
      H[(size_t)(k + 1) * m + k] = hn;
      if (!std::isfinite(hn)) {
        ns->status = LBO_ENAN;
        return LBO_ENAN;
      }
      if (hn > 0)
        LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(len), 256, 0, S->V + (size_t)(k + 1) * len, S->w,
                   1.0 / hn, 0.0, len);
      // Givens rotations
      for (int i = 0; i < k; ++i) {
        double a = H[(size_t)i * m + k], b = H[(size_t)(i + 1) * m + k];
        H[(size_t)i * m + k] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
      }
      double a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
      double rr = std::hypot(a, b);
      cs[k] = rr > 0 ? a / rr : 1.0;
      sn[k] = rr > 0 ? b / rr : 0.0;
      H[(size_t)k * m + k] = rr;
      H[(size_t)(k + 1) * m + k] = 0.0;
      gam[k + 1] = -sn[k] * gam[k];
      gam[k] = cs[k] * gam[k];
      ns->krylov_iterations++;
      if (std::fabs(gam[k + 1]) <= tol || hn == 0.0) {
        done = true;
        ++k;
        break;
      }
      if (ns->krylov_iterations >= S->pb.krylov_maxit) {
        done = true;
        ns->status = LBO_ENOTCONV;
        ++k;
        break;
      }
      if (learned && !S->force_sweep && ns->krylov_iterations >= learned_budget) {
        ++k;  // end this cycle; the restart below switches to the sweep
        break;
      }
    }
    // x += Z y,  H(0:k,0:k) y = gam(0:k)
    for (int i = k - 1; i >= 0; --i) {
      double acc = gam[i];
      for (int j = i + 1; j < k; ++j) acc -= H[(size_t)i * m + j] * y[j];
      y[i] = H[(size_t)i * m + i] != 0 ? acc / H[(size_t)i * m + i] : 0.0;
    }
    for (int i = 0; i < k; ++i) hv2[i] = -y[i];
    cudaMemcpyAsync(S->res + 8, hv2.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s);
    LBO_LAUNCH(S->plan, "solver_sub", s, k_sub_combination, grid_for(len), 256, 0, S->x, S->Z, len, k, S->res + 8, len);
    if (done) break;
    if (learned && !S->force_sweep && ns->krylov_iterations >= learned_budget) {
      S->force_sweep = true;
      ns->fallbacks++;
    }
    // restart from the true residual
    ns->restarts++;
    st = apply_op(S, S->x, S->w);
    if (st != LBO_OK) return st;
    cudaMemcpyAsync(S->V, S->rhs, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(len), 256, 0, S->V, S->w, -1.0, 1.0, len);
    beta = norm2(S, S->V, &st);
    if (st != LBO_OK) return st;
    if (beta <= tol) break;
  }
  return LBO_OK;
}

// ---------------------------------------------------------------------------
// Device-resident Arnoldi (problem.device_krylov = 1).  The Gram-Schmidt
// coefficients, the norms, the Givens rotations and the stopping test stay
// in device memory; a restart cycle is one eagerly launched iteration (it
// sizes every workspace of the operator) followed by a CUDA graph whose
// WHILE node repeats the iteration body until the device-side test clears
// its condition.  The host reads nothing inside a cycle: the cycle's
// status once at its end, and the restart residual norm.  The body reads
// the iteration index k from device memory, so one captured body serves
// every k (V_k and Z_k pass through two fixed vectors).  Same arithmetic as
// fgmres() above; scope: modified Jacobian, NONE / SWEEP preconditioners,
// uniform N, no training-pair collection.

struct DevArnoldi {
  double* H = nullptr;  // (m + 1) x m, then cs[m], sn[m], gam[m + 1], hv[m + 1], c[m], sc[4]
  double *cs = nullptr, *sn = nullptr, *gam = nullptr, *hv = nullptr, *c = nullptr, *sc = nullptr;
  int* ik = nullptr;       // k, iterations, status, k_used, continue, maxit
  int* host_ik = nullptr;  // pinned copy read at the end of a cycle
  double *vin = nullptr, *zbuf = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
};
enum { IK_K = 0, IK_ITS, IK_STATUS, IK_USED, IK_CONT, IK_MAXIT, IK_N };
enum { DS_RUNNING = 0, DS_CONVERGED = 1, DS_MAXIT = 2, DS_NAN = 3 };

// dst = base + (k + ofs) ld
__global__ void k_get_col(double* __restrict__ dst, const double* __restrict__ base, size_t ld,
                          const int* __restrict__ ik, int ofs, size_t len) {
  const double* src = base + (size_t)(ik[IK_K] + ofs) * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// base + (k + ofs) ld = src, or src / *hn when hn is given (left alone if *hn <= 0)
__global__ void k_put_col(double* __restrict__ base, size_t ld, const int* __restrict__ ik, int ofs,
                          const double* __restrict__ src, const double* __restrict__ hn, size_t len) {
  double a = 1.0;
  if (hn) {
    if (!(*hn > 0)) return;
    a = 1.0 / *hn;
  }
  double* dst = base + (size_t)(ik[IK_K] + ofs) * ld;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = hn ? src[e] * a : src[e];
}

// part[b K + i] = block b's share of <V_i, y>, K = *Kp + Kadd
__global__ void __launch_bounds__(RED_THREADS) k_dots_dev(const double* __restrict__ V, size_t ld,
                                                          const int* __restrict__ Kp, int Kadd,
                                                          const double* __restrict__ y, size_t len,
                                                          double* __restrict__ part) {
  __shared__ double sh[32];
  const int K = *Kp + Kadd;
  for (int k0 = 0; k0 < K; k0 += DOT_TILE) {
    double acc[DOT_TILE];
#pragma unroll
    for (int t = 0; t < DOT_TILE; ++t) acc[t] = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
      const double ye = y[e];
#pragma unroll
      for (int t = 0; t < DOT_TILE; ++t)
        if (k0 + t < K) acc[t] += V[(size_t)(k0 + t) * ld + e] * ye;
    }
#pragma unroll
    for (int t = 0; t < DOT_TILE; ++t) {
      double s = block_sum(acc[t], sh);
      if (threadIdx.x == 0 && k0 + t < K) part[blockIdx.x * K + k0 + t] = s;
    }
  }
}

// hv[i] = sum of the parts (fixed order), i <= k; column k of H set (pass 0) or
// increased (pass 1) by hv
__global__ void k_reduce_h(const double* __restrict__ part, int nb, const int* __restrict__ ik, double* __restrict__ hv,
                           double* __restrict__ H, int m, int pass) {
  const int k = ik[IK_K], K = k + 1;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b * K + i];
    hv[i] = s;
    H[(size_t)i * m + k] = pass == 0 ? s : H[(size_t)i * m + k] + s;
  }
}

// out = sqrt(sum of the parts)
__global__ void k_norm_finish(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = sqrt(s);
  }
}

// y -= sum_i c[i] V_i, i < *Kp + Kadd
__global__ void k_sub_comb_dev(double* __restrict__ y, const double* __restrict__ V, size_t ld,
                               const int* __restrict__ Kp, int Kadd, const double* __restrict__ c, size_t len) {
  const int K = *Kp + Kadd;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int k = 0; k < K; ++k) s += c[k] * V[(size_t)k * ld + e];
    y[e] -= s;
  }
}

// Start of a cycle: gam = beta e_0, k = 0, status running.
__global__ void k_cycle_init(double* __restrict__ gam, double* __restrict__ sc, int* __restrict__ ik, int m,
                             double beta, double tol, int iterations, int maxit) {
  for (int i = threadIdx.x; i <= m; i += blockDim.x) gam[i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    sc[1] = tol;
    ik[IK_K] = 0;
    ik[IK_ITS] = iterations;
    ik[IK_STATUS] = DS_RUNNING;
    ik[IK_USED] = 0;
    ik[IK_CONT] = 0;
    ik[IK_MAXIT] = maxit;
  }
}

// H(k+1, k) = hn, the earlier rotations and a new one on column k, the
// residual estimate gam(k+1) against tol; decides whether the cycle goes on
// (condition of the WHILE node when launched inside the graph).
__global__ void k_givens(double* __restrict__ H, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ gam, const double* __restrict__ sc, int* __restrict__ ik, int m,
                         cudaGraphConditionalHandle cond, int in_graph) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = ik[IK_K];
  const double hn = sc[2], tol = sc[1];
  int cont = 0;
  H[(size_t)(k + 1) * m + k] = hn;
  if (!isfinite(hn)) {
    ik[IK_STATUS] = DS_NAN;
    ik[IK_USED] = k;
  } else {
    for (int i = 0; i < k; ++i) {
      const double a = H[(size_t)i * m + k], b = H[(size_t)(i + 1) * m + k];
      H[(size_t)i * m + k] = cs[i] * a + sn[i] * b;
      H[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
    }
    const double a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
    const double rr = hypot(a, b);
    cs[k] = rr > 0 ? a / rr : 1.0;
    sn[k] = rr > 0 ? b / rr : 0.0;
    H[(size_t)k * m + k] = rr;
    H[(size_t)(k + 1) * m + k] = 0.0;
    gam[k + 1] = -sn[k] * gam[k];
    gam[k] = cs[k] * gam[k];
    const int its = ++ik[IK_ITS];
    if (fabs(gam[k + 1]) <= tol || hn == 0.0) {
      ik[IK_STATUS] = DS_CONVERGED;
      ik[IK_USED] = k + 1;
    } else if (its >= ik[IK_MAXIT]) {
      ik[IK_STATUS] = DS_MAXIT;
      ik[IK_USED] = k + 1;
    } else if (k + 1 == m) {
      ik[IK_USED] = m;
    } else {
      cont = 1;
      ik[IK_K] = k + 1;
    }
  }
  ik[IK_CONT] = cont;
  if (in_graph) cudaGraphSetConditional(cond, cont);
}

// first node of the cycle graph: the WHILE condition from the eager iteration
__global__ void k_set_cond(cudaGraphConditionalHandle cond, const int* __restrict__ ik) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(cond, ik[IK_CONT]);
}

// c = -y with H(0:k, 0:k) y = gam(0:k), k = ik[IK_USED] (back substitution)
__global__ void k_backsolve(const double* __restrict__ H, const double* __restrict__ gam, double* __restrict__ c,
                            const int* __restrict__ ik, int m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = ik[IK_USED];
  for (int i = k - 1; i >= 0; --i) {
    double acc = gam[i];
    for (int j = i + 1; j < k; ++j) acc += H[(size_t)i * m + j] * c[j];  // c holds -y
    c[i] = H[(size_t)i * m + i] != 0 ? -acc / H[(size_t)i * m + i] : 0.0;
  }
}

lbo_status dev_alloc(lbo_solver* S, DevArnoldi** out) {
  if (S->devk) {
    *out = (DevArnoldi*)S->devk;
    return LBO_OK;
  }
  DevArnoldi* D = new DevArnoldi();
  const int m = S->m;
  const size_t nsmall = (size_t)(m + 1) * m + m + m + (m + 1) + (m + 1) + m + 4;
  cudaError_t e = cudaMalloc(&D->H, sizeof(double) * nsmall);
  if (e == cudaSuccess) e = cudaMalloc(&D->ik, sizeof(int) * IK_N);
  if (e == cudaSuccess) e = cudaMallocHost(&D->host_ik, sizeof(int) * IK_N);
  if (e == cudaSuccess) e = cudaMalloc(&D->vin, sizeof(double) * S->len);
  if (e == cudaSuccess) e = cudaMalloc(&D->zbuf, sizeof(double) * S->len);
  S->devk = D;  // freed with the solver, also on failure
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error_text("device Krylov buffers");
    return LBO_ENOMEM;
  }
  D->cs = D->H + (size_t)(m + 1) * m;
  D->sn = D->cs + m;
  D->gam = D->sn + m;
  D->hv = D->gam + (m + 1);
  D->c = D->hv + (m + 1);
  D->sc = D->c + m;
  *out = D;
  return LBO_OK;
}

void dev_drop_graph(DevArnoldi* D) {
  if (D->exec) cudaGraphExecDestroy(D->exec);
  if (D->graph) cudaGraphDestroy(D->graph);
  D->exec = nullptr;
  D->graph = nullptr;
}

// One Arnoldi iteration on device state (k read from device memory).
lbo_status dev_iteration(lbo_solver* S, DevArnoldi* D, int in_graph) {
  cudaStream_t s = S->plan->stream;
  const size_t len = S->len;
  const int m = S->m;
  LBO_LAUNCH(S->plan, "krylov_get", s, k_get_col, grid_for(len), 256, 0, D->vin, S->V, len, D->ik, 0, len);
  lbo_status st = apply_precond(S, D->vin, D->zbuf);
  if (st != LBO_OK) return st;
  LBO_LAUNCH(S->plan, "krylov_put", s, k_put_col, grid_for(len), 256, 0, S->Z, len, D->ik, 0, D->zbuf,
             (const double*)nullptr, len);
  st = apply_op(S, D->zbuf, S->w);
  if (st != LBO_OK) return st;
  for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, two passes, FP64
    LBO_LAUNCH(S->plan, "krylov_dots", s, k_dots_dev, RED_BLOCKS, RED_THREADS, 0, S->V, len, D->ik + IK_K, 1,
               S->w, len, S->part);
    LBO_LAUNCH(S->plan, "krylov_reduce_h", s, k_reduce_h, 1, 256, 0, S->part, RED_BLOCKS, D->ik, D->hv, D->H, m,
               pass);
    LBO_LAUNCH(S->plan, "krylov_sub", s, k_sub_comb_dev, grid_for(len), 256, 0, S->w, S->V, len, D->ik + IK_K, 1,
               D->hv, len);
  }
  LBO_LAUNCH(S->plan, "krylov_dots", s, k_dots, RED_BLOCKS, RED_THREADS, 0, S->w, (size_t)0, 1, S->w, len,
             S->part);
  LBO_LAUNCH(S->plan, "krylov_norm", s, k_norm_finish, 1, 32, 0, S->part, RED_BLOCKS, D->sc + 2);
  LBO_LAUNCH(S->plan, "krylov_put", s, k_put_col, grid_for(len), 256, 0, S->V, len, D->ik, 1, S->w,
             (const double*)(D->sc + 2), len);
  LBO_LAUNCH(S->plan, "krylov_givens", s, k_givens, 1, 32, 0, D->H, D->cs, D->sn, D->gam, D->sc, D->ik, m, D->cond,
             in_graph);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "device Arnoldi iteration");
}

// The cycle graph [k_set_cond] -> WHILE { dev_iteration }, captured on a
// private stream (the plan's may be the legacy default stream) and
// instantiated; kernel parameters (shift, the cached Maxwellians, buffers)
// are those of the current Newton step.
lbo_status dev_capture(lbo_solver* S, DevArnoldi* D) {
  dev_drop_graph(D);
  cudaError_t e = cudaGraphCreate(&D->graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&D->cond, D->graph, 0, 0);
  cudaGraphNode_t n_set = nullptr, n_loop = nullptr;
  if (e == cudaSuccess) {
    void* args[] = {(void*)&D->cond, (void*)&D->ik};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_set_cond;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&n_set, D->graph, nullptr, 0, &kp);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = D->cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&n_loop, D->graph, &n_set, nullptr, 1, &cp);
  cudaStream_t cap = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    dev_drop_graph(D);
    return cuda_fail(e, "device Krylov graph");
  }
  cudaStream_t own = S->plan->stream;
  S->plan->stream = cap;
  lbo_status st = LBO_OK;
  e = cudaStreamBeginCaptureToGraph(cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = dev_iteration(S, D, 1);
    cudaGraph_t body = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &body);
    if (st == LBO_OK && e2 != cudaSuccess) e = e2;
  }
  S->plan->stream = own;
  cudaStreamDestroy(cap);
  if (e == cudaSuccess && st == LBO_OK) e = cudaGraphInstantiate(&D->exec, D->graph, 0);
  if (e != cudaSuccess || st != LBO_OK) {
    cudaGetLastError();
    dev_drop_graph(D);
    return st != LBO_OK ? st : cuda_fail(e, "device Krylov graph capture");
  }
  return LBO_OK;
}

// Restarted FGMRES with the device-resident Arnoldi: same iteration and
// stopping tests as fgmres(), host reads only at the ends of cycles.
lbo_status fgmres_device(lbo_solver* S, lbo_newton_stats* ns) {
  DevArnoldi* D = nullptr;
  lbo_status st = dev_alloc(S, &D);
  if (st != LBO_OK) return st;
  const size_t len = S->len;
  cudaStream_t s = S->plan->stream;
  cudaMemsetAsync(S->x, 0, sizeof(double) * len, s);
  double rhs_norm = norm2(S, S->rhs, &st);
  if (st != LBO_OK) return st;
  ns->rhs_norm = rhs_norm * std::sqrt(S->wnorm);
  const double tol = std::fmax(S->pb.krylov_rtol * rhs_norm, S->pb.krylov_atol / std::sqrt(S->wnorm));
  ns->krylov_iterations = 0;
  ns->restarts = 0;
  ns->status = LBO_OK;
  if (rhs_norm == 0.0) return LBO_OK;
  if (!std::isfinite(rhs_norm)) {
    ns->status = LBO_ENAN;
    return LBO_ENAN;
  }
  cudaMemcpyAsync(S->V, S->rhs, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
  double beta = rhs_norm;
  bool captured = false;
  for (;;) {
    LBO_LAUNCH(S->plan, "solver_scale", s, k_scale, grid_for(len), 256, 0, S->V, 1.0 / beta, len);
    cudaMemsetAsync(D->H, 0, sizeof(double) * (size_t)(S->m + 1) * S->m, s);
    LBO_LAUNCH(S->plan, "krylov_init", s, k_cycle_init, 1, 256, 0, D->gam, D->sc, D->ik, S->m, beta, tol,
               ns->krylov_iterations, S->pb.krylov_maxit);
    st = dev_iteration(S, D, 0);  // k = 0, eagerly: sizes the operator's workspaces
    if (st != LBO_OK) return st;
    if (!captured) {
      st = dev_capture(S, D);
      if (st != LBO_OK) return st;
      captured = true;
    }
    cudaError_t e = cudaGraphLaunch(D->exec, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D->host_ik, D->ik, sizeof(int) * IK_N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device Krylov cycle");
    ns->krylov_iterations = D->host_ik[IK_ITS];
    const int status = D->host_ik[IK_STATUS];
    if (status == DS_NAN) {
      ns->status = LBO_ENAN;
      return LBO_ENAN;
    }
    // x += Z y,  H(0:k,0:k) y = gam(0:k)
    LBO_LAUNCH(S->plan, "krylov_backsolve", s, k_backsolve, 1, 32, 0, D->H, D->gam, D->c, D->ik, S->m);
    LBO_LAUNCH(S->plan, "krylov_sub", s, k_sub_comb_dev, grid_for(len), 256, 0, S->x, S->Z, len, D->ik + IK_USED, 0,
               D->c, len);
    if (status == DS_CONVERGED) break;
    if (status == DS_MAXIT) {
      ns->status = LBO_ENOTCONV;
      break;
    }
    // restart from the true residual
    ns->restarts++;
    st = apply_op(S, S->x, S->w);
    if (st != LBO_OK) return st;
    cudaMemcpyAsync(S->V, S->rhs, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(len), 256, 0, S->V, S->w, -1.0, 1.0, len);
    beta = norm2(S, S->V, &st);
    if (st != LBO_OK) return st;
    if (beta <= tol) break;
  }
  return LBO_OK;
}

bool device_krylov_applies(const lbo_solver* S) {
  return S->pb.device_krylov == 1 && !S->mixed && S->pb.jacobian == 0 && !S->plan->profiling &&
         (S->pb.precond == LBO_PRECOND_NONE || S->pb.precond == LBO_PRECOND_SWEEP) && !network_collecting(S);
}

// Source iteration (Sec. 5.2 and the supplement's discrete form): with S the
// operator of the upwind sweep, S g_{l+1} = (S - A) g_l + rhs from g_0 = 0,
// i.e. the Richardson iteration g += P(rhs - A g) with P the preconditioner
// (the sweep; with MOMENT or LEARNED also their corrections).  One operator
// and one preconditioner application per iteration, like an FGMRES step
// without the orthogonalisation; the FP64 residual decides convergence.
lbo_status source_iteration(lbo_solver* S, lbo_newton_stats* ns) {
  const size_t len = S->len;
  cudaStream_t s = S->plan->stream;
  lbo_status st;
  cudaMemsetAsync(S->x, 0, sizeof(double) * len, s);
  const double rhs_norm = norm2(S, S->rhs, &st);
  if (st != LBO_OK) return st;
  ns->rhs_norm = rhs_norm * std::sqrt(S->wnorm);
  const double tol = std::fmax(S->pb.krylov_rtol * rhs_norm, S->pb.krylov_atol / std::sqrt(S->wnorm));
  ns->krylov_iterations = 0;
  ns->restarts = 0;
  ns->status = LBO_OK;
  S->force_sweep = false;
  if (rhs_norm == 0.0) return LBO_OK;
  if (!std::isfinite(rhs_norm)) {
    ns->status = LBO_ENAN;
    return LBO_ENAN;
  }
  double* r = S->V;  // the residual rhs - A g, first rhs itself
  cudaMemcpyAsync(r, S->rhs, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
  for (;;) {
    st = apply_precond(S, r, S->Z);
    if (st != LBO_OK) return st;
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(len), 256, 0, S->x, S->Z, 1.0, 1.0, len);
    ns->krylov_iterations++;
    st = apply_op(S, S->x, S->w);
    if (st != LBO_OK) return st;
    cudaMemcpyAsync(r, S->rhs, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(len), 256, 0, r, S->w, -1.0, 1.0, len);
    const double rn = norm2(S, r, &st);
    if (st != LBO_OK) return st;
    if (!std::isfinite(rn)) {
      ns->status = LBO_ENAN;
      return LBO_ENAN;
    }
    if (rn <= tol) return LBO_OK;
    if (ns->krylov_iterations >= S->pb.krylov_maxit) {
      ns->status = LBO_ENOTCONV;
      return LBO_OK;
    }
  }
}

}  // namespace

double solver_norm2(lbo_solver* S, const double* y, lbo_status* st) { return norm2(S, y, st); }

lbo_status solver_sweep_uniform(lbo_solver* S, const double* r, double* z, int N, double h) {
  LBO_LAUNCH(S->plan, "solver_sweep", S->plan->stream, k_sweep, grid_for((size_t)N * N * N), 256, 0, r, z, S->nu, N,
             S->nx, h, S->dx, S->pb.kn, S->shift);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "sweep");
}

lbo_status solver_apply_op(lbo_solver* S, const double* v, double* out, bool border, bool collisions) {
  return apply_op(S, v, out, border, collisions);
}

void solver_axpby(lbo_solver* S, double* y, const double* x, double a, double b) {
  LBO_LAUNCH(S->plan, "solver_axpby", S->plan->stream, k_axpby, grid_for(S->len), 256, 0, y, x, a, b, S->len);
}


namespace {
lbo_status apply_precond(lbo_solver* S, const double* v, double* z) {
  cudaStream_t s = S->plan->stream;
  const int pc = S->pb.precond;
  if (pc == LBO_PRECOND_NONE || S->pb.kind != LBO_PROBLEM_SLAB) {
    cudaMemcpyAsync(z, v, sizeof(double) * S->len, cudaMemcpyDeviceToDevice, s);
  } else {
    if (S->mixed) {
      lbo_status st = mixed_sweep(S, v, z);
      if (st != LBO_OK) return st;
    } else {
      LBO_LAUNCH(S->plan, "solver_sweep", s, k_sweep, grid_for(S->n3), 256, 0, v, z, S->nu, S->N, S->nx, S->h,
                 S->dx, S->pb.kn, S->shift);
    }
    if (pc == LBO_PRECOND_LEARNED && !S->force_sweep) {
      lbo_status st = network_correction(S, v, z);
      if (st != LBO_OK) return st;
    }
    if (pc == LBO_PRECOND_MOMENT) {
      lbo_status st = coarse_correct(S, v, z);
      if (st != LBO_OK) return st;
    }
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "preconditioner");
}
}  // namespace

}  // namespace lbo

using namespace lbo;

// Krylov basis and work vectors of S->len doubles, small reduction buffers.
static lbo_status solver_alloc(lbo_solver* S) {
  const lbo_problem* pb = &S->pb;
  const size_t len = S->len;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double** p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(p, sizeof(double) * n);
  };
  alloc(&S->V, (size_t)(S->m + 1) * len);
  alloc(&S->Z, (size_t)S->m * len);
  alloc(&S->w, len);
  alloc(&S->Lv, len);
  alloc(&S->rhs, len);
  alloc(&S->x, len);
  alloc(&S->evec, len);
  if (pb->jacobian == 1) {
    alloc(&S->ja, len);
    alloc(&S->jb, len);
  }
  alloc(&S->Qf, len);
  alloc(&S->params, 5 * (size_t)S->nx);
  alloc(&S->nu, S->nx);
  alloc(&S->WL, S->n3);
  alloc(&S->WR, S->n3);
  alloc(&S->part, (size_t)RED_BLOCKS * 256);
  alloc(&S->res, 8 + 256);
  if (e == cudaSuccess) e = cudaMallocHost(&S->host, sizeof(double) * 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lbo_solver_destroy(S);
    set_error_text("solver allocation");
    return LBO_ENOMEM;
  }
  return LBO_OK;
}

extern "C" {

lbo_status lbo_solver_create(const lbo_problem* pb, lbo_plan* plan, lbo_solver** out) {
  if (!pb || !plan || !out) return LBO_EINVAL;
  *out = nullptr;
  if (pb->nx < 1 || pb->krylov_restart < 1 || pb->krylov_restart > 200 || pb->krylov_maxit < 1) return LBO_EINVAL;
  if (pb->kind == LBO_PROBLEM_SLAB) {
    if (!(pb->x_right > pb->x_left) || !(pb->kn > 0) || !(pb->total_mass > 0)) return LBO_EINVAL;
    for (int side = 0; side < 2; ++side) {
      const int bc = side == 0 ? pb->bc_left : pb->bc_right;
      const double* w = side == 0 ? pb->wall_left : pb->wall_right;
      const double* in = side == 0 ? pb->inflow_left : pb->inflow_right;
      if (bc == LBO_BC_WALL) {
        if (!(w[0] > 0) || w[1] != 0.0) return LBO_EINVAL;
      } else if (bc == LBO_BC_INFLOW) {
        if (!(in[0] > 0) || !(in[4] > 0)) return LBO_EINVAL;
      } else {
        return LBO_EINVAL;
      }
    }
  } else if (pb->kind == LBO_PROBLEM_HOMOGENEOUS) {
    if (!(pb->dt > 0)) return LBO_EINVAL;
  } else {
    return LBO_EINVAL;
  }
  if (pb->precond < 0 || pb->precond > 3) return LBO_EINVAL;
  if (pb->line_search < 0 || pb->line_search > 60 || !(pb->pseudo_dt >= 0)) return LBO_EINVAL;
  if (pb->jacobian < 0 || pb->jacobian > 1 || pb->device_krylov < 0 || pb->device_krylov > 1) return LBO_EINVAL;
  if (pb->coarse_operator < 0 || pb->coarse_operator > 1) return LBO_EINVAL;
  if (pb->inner_solver < 0 || pb->inner_solver > 1 || !(pb->nu_scale >= 0) || !std::isfinite(pb->nu_scale))
    return LBO_EINVAL;
  if (pb->inner_solver == 1 && (pb->kind != LBO_PROBLEM_SLAB || pb->precond == LBO_PRECOND_NONE)) return LBO_EINVAL;
  lbo_solver* S = new lbo_solver();
  S->pb = *pb;
  S->plan = plan;
  S->N = plan->N;
  S->nx = pb->nx;
  S->m = pb->krylov_restart;
  S->n3 = (size_t)S->N * S->N * S->N;
  S->len = S->n3 * S->nx;
  S->h = 2.0 * plan->L / S->N;
  S->dx = pb->kind == LBO_PROBLEM_SLAB ? (pb->x_right - pb->x_left) / pb->nx : 1.0;
  S->wnorm = S->dx * S->h * S->h * S->h;
  lbo_status ast = solver_alloc(S);
  if (ast != LBO_OK) return ast;
  if (pb->kind == LBO_PROBLEM_SLAB) {
    // wall Maxwellian shapes W(v) = (2 pi theta)^{-3/2} exp(-|v-u_w|^2 / (2 theta))
    std::vector<double> wl(S->n3), wr(S->n3);
    const int N = S->N;
    double sumL = 0, sumR = 0;
    for (size_t k = 0; k < S->n3; ++k) {
      const int i1 = (int)(k / ((size_t)N * N)), i2 = (int)((k / N) % N), i3 = (int)(k % N);
      const double v[3] = {(i1 - N / 2) * S->h, (i2 - N / 2) * S->h, (i3 - N / 2) * S->h};
      for (int side = 0; side < 2; ++side) {
        const bool inflow = (side == 0 ? pb->bc_left : pb->bc_right) == LBO_BC_INFLOW;
        const double* wp = side == 0 ? pb->wall_left : pb->wall_right;
        const double* in = side == 0 ? pb->inflow_left : pb->inflow_right;
        // wall: unit-density Maxwellian (theta_w, u_w); inflow: the given state
        const double th = inflow ? in[4] : wp[0], rho = inflow ? in[0] : 1.0;
        const double* u = inflow ? in + 1 : wp + 1;
        const double d2 = (v[0] - u[0]) * (v[0] - u[0]) + (v[1] - u[1]) * (v[1] - u[1]) +
                          (v[2] - u[2]) * (v[2] - u[2]);
        const double W = rho * std::pow(2.0 * 3.141592653589793 * th, -1.5) * std::exp(-d2 / (2.0 * th));
        (side == 0 ? wl : wr)[k] = W;
      }
      if (v[0] > 0) sumL += v[0] * wl[k];
      if (v[0] < 0) sumR -= v[0] * wr[k];
    }
    const double h3 = S->h * S->h * S->h;
    if (pb->wall_flux == LBO_WALL_FLUX_DISCRETE) {
      S->kL = 1.0 / (h3 * sumL);
      S->kR = 1.0 / (h3 * sumR);
    } else {
      S->kL = pb->bc_left == LBO_BC_WALL ? std::sqrt(2.0 * 3.141592653589793 / pb->wall_left[0]) : 0.0;
      S->kR = pb->bc_right == LBO_BC_WALL ? std::sqrt(2.0 * 3.141592653589793 / pb->wall_right[0]) : 0.0;
    }
    cudaError_t e = cudaMemcpy(S->WL, wl.data(), sizeof(double) * S->n3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(S->WR, wr.data(), sizeof(double) * S->n3, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      lbo_solver_destroy(S);
      return cuda_fail(e, "solver tables");
    }
  }
  *out = S;
  return LBO_OK;
}

lbo_status lbo_solver_create_mixed(const lbo_problem* pb, lbo_plan* const* plans, int nplans, const int* cell_plan,
                                   lbo_solver** out) {
  if (!pb || !plans || nplans < 1 || !cell_plan || !out) return LBO_EINVAL;
  *out = nullptr;
  if (pb->kind != LBO_PROBLEM_SLAB || pb->nx < 1 || pb->krylov_restart < 1 || pb->krylov_restart > 200 ||
      pb->krylov_maxit < 1 || !(pb->x_right > pb->x_left) || !(pb->kn > 0))
    return LBO_EINVAL;
  if (pb->bc_left != LBO_BC_INFLOW || pb->bc_right != LBO_BC_INFLOW) return LBO_EUNSUPPORTED;
  if (!(pb->inflow_left[0] > 0) || !(pb->inflow_left[4] > 0) || !(pb->inflow_right[0] > 0) ||
      !(pb->inflow_right[4] > 0))
    return LBO_EINVAL;
  if (pb->precond != LBO_PRECOND_NONE && pb->precond != LBO_PRECOND_SWEEP) return LBO_EUNSUPPORTED;
  if (pb->line_search < 0 || pb->line_search > 60 || !(pb->pseudo_dt >= 0)) return LBO_EINVAL;
  if (pb->jacobian < 0 || pb->jacobian > 1) return LBO_EINVAL;
  if (pb->inner_solver < 0 || pb->inner_solver > 1 || !(pb->nu_scale >= 0) || !std::isfinite(pb->nu_scale))
    return LBO_EINVAL;
  if (pb->inner_solver == 1 && pb->precond == LBO_PRECOND_NONE) return LBO_EINVAL;
  int nmax = 0;
  for (int p = 0; p < nplans; ++p) {
    if (!plans[p] || plans[p]->L != plans[0]->L || plans[p]->N > 64) return LBO_EINVAL;
    for (int q = 0; q < p; ++q)
      if (plans[q]->N == plans[p]->N) return LBO_EINVAL;  // one plan per N
    nmax = std::max(nmax, plans[p]->N);
  }
  for (int j = 0; j < pb->nx; ++j)
    if (cell_plan[j] < 0 || cell_plan[j] >= nplans) return LBO_EINVAL;
  lbo_solver* S = new lbo_solver();
  S->pb = *pb;
  S->plan = plans[0];  // the stream and profiling scope of the solver's own launches
  S->N = nmax;
  S->nx = pb->nx;
  S->m = pb->krylov_restart;
  S->n3 = (size_t)nmax * nmax * nmax;
  S->len = mixed_state_length(plans, pb->nx, cell_plan);
  S->h = 2.0 * plans[0]->L / nmax;
  S->dx = (pb->x_right - pb->x_left) / pb->nx;
  S->wnorm = S->dx * S->h * S->h * S->h;  // finest cell's weight, for the absolute tolerance only
  lbo_status st = solver_alloc(S);
  if (st != LBO_OK) return st;
  st = mixed_setup(S, plans, nplans, cell_plan);
  if (st != LBO_OK) {
    lbo_solver_destroy(S);
    return st;
  }
  *out = S;
  return LBO_OK;
}

size_t lbo_solver_state_length(const lbo_solver* S) { return S ? S->len : 0; }

lbo_status lbo_solver_residual(lbo_solver* S, const double* f, const double* f_prev, double* out, double* nrm) {
  if (!S || !f || !out) return LBO_EINVAL;
  if (S->pb.kind == LBO_PROBLEM_HOMOGENEOUS && !f_prev) return LBO_EINVAL;
  return residual(S, f, f_prev, out, nrm);
}

lbo_status lbo_solver_set_residual_plan(lbo_solver* S, lbo_plan* plan) {
  if (!S) return LBO_EINVAL;
  if (S->mixed) return mixed_set_residual_plan(S, plan);
  if (plan && (plan->N != S->plan->N || plan->L != S->plan->L)) return LBO_EINVAL;
  S->rplan = plan;
  return LBO_OK;
}

lbo_status lbo_newton_step(lbo_solver* S, double* f, const double* f_prev, lbo_newton_stats* stats) {
  if (!S || !f) return LBO_EINVAL;
  if (S->pb.kind == LBO_PROBLEM_HOMOGENEOUS && !f_prev) return LBO_EINVAL;
  lbo_newton_stats local{};
  lbo_newton_stats* ns = stats ? stats : &local;
  std::memset(ns, 0, sizeof(*ns));
  cudaStream_t s = S->plan->stream;
  cudaEvent_t t0, t1, t2;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventCreate(&t2);
  cudaEventRecord(t0, s);
  // local Maxwellians (FP64 moments) and the nonlinear residual
  if (S->mixed) mixed_moments(S, f, S->params, S->nu);
  else LBO_LAUNCH(S->plan, "solver_moments", s, k_cell_moments, S->nx, 512, 0, f, S->params, S->nu, S->N, S->h);
  if (S->pb.nu_scale > 0 && S->pb.nu_scale != 1.0)  // nu_j = nu_scale rho_j in the sweep
    LBO_LAUNCH(S->plan, "solver_scale", s, k_scale, grid_for(S->nx), 256, 0, S->nu, S->pb.nu_scale, (size_t)S->nx);
  double rn = 0;
  lbo_status st = residual(S, f, f_prev, S->rhs, &rn);
  cudaEventRecord(t1, s);
  if (st == LBO_OK && S->pb.jacobian == 1) {
    S->fcur = f;  // f stays unchanged until the linear solve is done
    S->fnorm = norm2(S, f, &st);
  }
  if (st == LBO_OK) {
    ns->residual_norm = rn;
    // pseudo-transient continuation: dtau = pseudo_dt |R_first| / |R_k|
    // (switched evolution relaxation); the shift 1/dtau fades as |R| falls
    S->shift = 0.0;
    if (S->pb.kind == LBO_PROBLEM_SLAB && S->pb.pseudo_dt > 0 && rn > 0) {
      if (S->r_first <= 0) S->r_first = rn;
      S->shift = rn / (S->pb.pseudo_dt * S->r_first);
    }
    ns->shift = S->shift;
    if (bordered(S)) {
      // bordered system: e = f / m(f), rhs = R + e (m(f) - C)
      wall_mass(S, f);
      double mf = 0;
      cudaError_t e = cudaMemcpyAsync(&mf, S->res + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "newton step: mass of the state");
      } else {
        LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, S->evec, f, 1.0 / mf, 0.0,
                   S->len);
        LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, S->rhs, S->evec,
                   mf - S->pb.total_mass, 1.0, S->len);
      }
    }
    // the Krylov products of this step share the cells' Maxwellians: their
    // u^_j and loss factor are computed once (dropped before f changes)
    if (st == LBO_OK && S->pb.jacobian == 0 && !S->mixed)
      st = lbo_plan_cache_maxwellians(S->plan, S->params, S->nx);
    if (st == LBO_OK && S->pb.kind == LBO_PROBLEM_SLAB && S->pb.precond == LBO_PRECOND_MOMENT) {
      // coarse operator about this step's cell parameters (and shift)
      st = coarse_assemble(S, bordered(S));
      if (st == LBO_OK && !coarse_valid(S)) ns->fallbacks++;  // singular: sweep alone
    }
    if (st == LBO_OK)
      st = S->pb.inner_solver == 1     ? source_iteration(S, ns)
           : device_krylov_applies(S) ? fgmres_device(S, ns)
                                      : fgmres(S, ns);
    if (st == LBO_OK || st == LBO_ENOTCONV) {
      // FP64 true residual of the linear system
      lbo_status st2 = apply_op(S, S->x, S->w);
      if (st2 == LBO_OK) {
        LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, S->w, S->rhs, 1.0, -1.0, S->len);
        double lr = norm2(S, S->w, &st2);
        ns->linear_residual = lr * std::sqrt(S->wnorm);
      }
      lbo_plan_cache_maxwellians(S->plan, nullptr, 0);  // S->params changes from here on
      // f <- f - lambda g; with line search, halve lambda until the residual
      // norm decreases by the Armijo factor (the trial residual lands in S->w)
      LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, f, S->x, -1.0, 1.0, S->len);
      double lambda = 1.0;
      for (int ls = 0; st2 == LBO_OK && ls < S->pb.line_search; ++ls) {
        if (S->mixed) mixed_moments(S, f, S->params, nullptr);
        else LBO_LAUNCH(S->plan, "solver_moments", s, k_cell_moments, S->nx, 512, 0, f, S->params,
                        (double*)nullptr, S->N, S->h);
        double rt = 0;
        st2 = residual(S, f, f_prev, S->w, &rt);
        if (st2 != LBO_OK) break;
        if (std::isfinite(rt) && rt <= (1.0 - 1e-4 * lambda) * rn) break;
        // back off: f += (lambda / 2) g
        LBO_LAUNCH(S->plan, "solver_axpby", s, k_axpby, grid_for(S->len), 256, 0, f, S->x, 0.5 * lambda, 1.0,
                   S->len);
        lambda *= 0.5;
      }
      ns->step_length = lambda;
      if (st2 != LBO_OK) st = st2;
    }
  }
  lbo_plan_cache_maxwellians(S->plan, nullptr, 0);
  cudaEventRecord(t2, s);
  cudaEventSynchronize(t2);
  float a = 0, b = 0;
  cudaEventElapsedTime(&a, t0, t1);
  cudaEventElapsedTime(&b, t1, t2);
  ns->ms_residual = a;
  ns->ms_linear = b;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaEventDestroy(t2);
  if (st == LBO_OK && ns->status != LBO_OK) return (lbo_status)ns->status;
  cudaError_t e = cudaGetLastError();
  if (st == LBO_OK && e != cudaSuccess) return cuda_fail(e, "newton step");
  return st;
}

void lbo_solver_destroy(lbo_solver* S) {
  if (!S) return;
  double* bufs[] = {S->V,      S->Z,  S->w,  S->Lv, S->rhs, S->x,    S->evec, S->ja,
                    S->jb,     S->Qf, S->params, S->nu, S->WL,  S->WR, S->part, S->res};
  for (double* p : bufs)
    if (p) cudaFree(p);
  if (S->devk) {
    DevArnoldi* D = (DevArnoldi*)S->devk;
    dev_drop_graph(D);
    if (D->H) cudaFree(D->H);
    if (D->ik) cudaFree(D->ik);
    if (D->host_ik) cudaFreeHost(D->host_ik);
    if (D->vin) cudaFree(D->vin);
    if (D->zbuf) cudaFree(D->zbuf);
    delete D;
  }
  free_network(S);
  free_coarse(S);
  free_mixed(S);
  if (S->host) cudaFreeHost(S->host);
  delete S;
}

}  // extern "C"

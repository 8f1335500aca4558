// Mixed-N slab: every cell carries its own velocity grid (N in the plans'
// set) on the same box [-L, L)^3 -- the shock workload with a grid per cell;
// not in the paper, which uses one N everywhere.
//
// The state is the cells' fields concatenated, cell j holding N_j^3 values
// in centred order at offset off_j.  Collisions are cell-local: the cells of
// one N are gathered into a contiguous batch, the plan of that N applies L
// (or Q), and the results are scattered back.  The upwind difference of cell
// j needs its neighbours on its own grid: a neighbour of another N is
// spectrally resampled (reading: the field's trigonometric interpolant, the
// Nyquist term a cosine split between +-N/2; zero padding to a finer grid,
// truncation to a coarser one, where the pair +-N_b/2 coincides).  One
// axis of that resampling is the dense real matrix
//   R[b][a] = (1/N_a) [ sum_{|k| < K} cos(pi k (v_b - v_a) / L)
//                       + c cos(pi K v_a / L) cos(pi K v_b / L) ],
// K = min(N_a, N_b) / 2, c = 1 for padding and 2 for truncation, applied to
// the three axes in turn (one CTA per resampling job).  The residual
// resamples in FP64, the Krylov products in the plans' precision, the sweep
// in FP32.  The sweep
// preconditioner runs on the finest grid: every cell is resampled to it,
// swept with the uniform kernel, and resampled back.
// Scope: slab with inflow sides on both ends; preconditioner none or sweep;
// modified or exact Jacobian; pseudo-transient continuation; a residual plan
// per N.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "lbo_internal.h"

namespace lbo {
namespace {

constexpr int RT = 256;
constexpr int NMAXR = 64;

struct Group {
  lbo_plan* plan = nullptr;
  lbo_plan* rplan = nullptr;  // residual plan of this N, if set
  int N = 0;
  std::vector<int> cells;
  int* d_cells = nullptr;
  double* in = nullptr;      // gathered cells, count * N^3
  double* out = nullptr;     // plan output, count * N^3
  double* params = nullptr;  // gathered local Maxwellians, count * 5
};

// One resampling: src + src_off (N_a^3) -> dst + dst_off (N_b^3); mat is the
// offset of the N_b x N_a matrix; tmp the offset of two scratch cubes.
struct RJob {
  size_t src_off, dst_off, tmp_off;
  int na, nb, mat;
};

struct JobList {
  std::vector<RJob> host;
  RJob* dev = nullptr;
};

struct MixedState {
  int nx = 0, nmax = 0;
  double L = 0;
  std::vector<int> Nc;
  std::vector<size_t> off;
  int* d_N = nullptr;
  size_t* d_off = nullptr;
  std::vector<Group> groups;
  double* nb2 = nullptr;          // neighbours on the cell's grid: left [0, len), right [len, 2 len)
  double* gL = nullptr;           // inflow Maxwellian on the first cell's grid
  double* gR = nullptr;           // and on the last cell's
  double* mats64 = nullptr;       // resampling matrices
  float* mats32 = nullptr;
  double* tmp = nullptr;          // two scratch cubes per job
  double* sweep_in = nullptr;     // nx * nmax^3
  double* sweep_out = nullptr;
  JobList transport, to_max, from_max;
  size_t len = 0;
};

MixedState* mstate(lbo_solver* S) { return static_cast<MixedState*>(S->mixed); }

// ------------------------------------------------------------ kernels
template <typename TC>
__global__ void __launch_bounds__(RT) k_resample_jobs(const RJob* __restrict__ jobs, const double* __restrict__ src,
                                                      double* __restrict__ dst, const TC* __restrict__ mats,
                                                      double* __restrict__ tmp, size_t cube) {
  __shared__ TC R[NMAXR * NMAXR];
  const RJob jb = jobs[blockIdx.x];
  const int na = jb.na, nb = jb.nb, t = threadIdx.x;
  const double* s = src + jb.src_off;
  double* d = dst + jb.dst_off;
  if (na == nb) {  // same grid: copy
    for (size_t i = t; i < (size_t)na * na * na; i += RT) d[i] = s[i];
    return;
  }
  for (int i = t; i < na * nb; i += RT) R[i] = mats[jb.mat + i];
  __syncthreads();
  double* t1 = tmp + jb.tmp_off;                       // [a1][a2][b3]
  double* t2 = t1 + cube;                              // [a1][b2][b3]
  for (size_t idx = t; idx < (size_t)na * na * nb; idx += RT) {
    const int b3 = (int)(idx % nb);
    const double* x = s + (idx / nb) * na;
    TC acc = 0;
    for (int a = 0; a < na; ++a) acc += R[b3 * na + a] * (TC)x[a];
    t1[idx] = (double)acc;
  }
  __syncthreads();
  for (size_t idx = t; idx < (size_t)na * nb * nb; idx += RT) {
    const int b3 = (int)(idx % nb), b2 = (int)((idx / nb) % nb);
    const size_t a1 = idx / ((size_t)nb * nb);
    TC acc = 0;
    for (int a = 0; a < na; ++a) acc += R[b2 * na + a] * (TC)t1[(a1 * na + a) * nb + b3];
    t2[idx] = (double)acc;
  }
  __syncthreads();
  for (size_t idx = t; idx < (size_t)nb * nb * nb; idx += RT) {
    const size_t b23 = idx % ((size_t)nb * nb);
    const int b1 = (int)(idx / ((size_t)nb * nb));
    TC acc = 0;
    for (int a = 0; a < na; ++a) acc += R[b1 * na + a] * (TC)t2[a * (size_t)nb * nb + b23];
    d[idx] = (double)acc;
  }
}

// cells listed in `cells` between the concatenated layout and a batch
__global__ void k_gather(const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ cells,
                         const size_t* __restrict__ off, size_t n3, int to_batch) {
  const int slot = blockIdx.y;
  const size_t o = off[cells[slot]];
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n3; k += (size_t)gridDim.x * blockDim.x) {
    if (to_batch) dst[slot * n3 + k] = src[o + k];
    else dst[o + k] = src[slot * n3 + k];
  }
}

__global__ void k_gather_params(const double* __restrict__ params, double* __restrict__ out,
                                const int* __restrict__ cells, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 5 * count) out[i] = params[5 * cells[i / 5] + i % 5];
}

// local Maxwellian of each cell (rho, u, theta), FP64, cell j on its own grid
__global__ void __launch_bounds__(256) k_mixed_moments(const double* __restrict__ f, const int* __restrict__ Nc,
                                                       const size_t* __restrict__ off, double L,
                                                       double* __restrict__ params, double* __restrict__ nu) {
  __shared__ double sh[5][8];
  __shared__ double mom[4];
  const int j = blockIdx.x, N = Nc[j], t = threadIdx.x, lane = t & 31, w = t >> 5;
  const size_t n3 = (size_t)N * N * N;
  const double h = 2.0 * L / N;
  const double* x = f + off[j];
  double m[4] = {0, 0, 0, 0};
  for (size_t k = t; k < n3; k += 256) {
    const int i3 = (int)(k % N), i2 = (int)((k / N) % N), i1 = (int)(k / ((size_t)N * N));
    const double y = x[k];
    m[0] += y;
    m[1] += (i1 - N / 2) * h * y;
    m[2] += (i2 - N / 2) * h * y;
    m[3] += (i3 - N / 2) * h * y;
  }
  for (int a = 0; a < 4; ++a) {
    double v = m[a];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[a][w] = v;
  }
  __syncthreads();
  if (t < 4) {
    double v = 0;
    for (int i = 0; i < 8; ++i) v += sh[t][i];
    mom[t] = v;
  }
  __syncthreads();
  const double h3 = h * h * h, rho = h3 * mom[0];
  const double u1 = h3 * mom[1] / rho, u2 = h3 * mom[2] / rho, u3 = h3 * mom[3] / rho;
  double e = 0;
  for (size_t k = t; k < n3; k += 256) {
    const int i3 = (int)(k % N), i2 = (int)((k / N) % N), i1 = (int)(k / ((size_t)N * N));
    const double c1 = (i1 - N / 2) * h - u1, c2 = (i2 - N / 2) * h - u2, c3 = (i3 - N / 2) * h - u3;
    e += (c1 * c1 + c2 * c2 + c3 * c3) * x[k];
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if (lane == 0) sh[4][w] = e;
  __syncthreads();
  if (t == 0) {
    double v = 0;
    for (int i = 0; i < 8; ++i) v += sh[4][i];
    double* p = params + 5 * j;
    p[0] = rho;
    p[1] = u1;
    p[2] = u2;
    p[3] = u3;
    p[4] = h3 * v / (3.0 * rho);
    if (nu) nu[j] = rho;
  }
}

// out = cT (v1^+ (v - left) + v1^- (right - v)) / dx + cY y + cV v per cell,
// neighbours of another N taken from nb (resampled), inflow ghosts gs * g
__global__ void k_mixed_transport(const double* __restrict__ v, const double* __restrict__ y,
                                  const double* __restrict__ nb, size_t len, const double* __restrict__ gL,
                                  const double* __restrict__ gR, double* __restrict__ out,
                                  const int* __restrict__ Nc, const size_t* __restrict__ off, int nx, double L,
                                  double dx, double cT, double cY, double gs, double cV) {
  const int j = blockIdx.y, N = Nc[j];
  const size_t n3 = (size_t)N * N * N, o = off[j];
  const double h = 2.0 * L / N;
  const bool sameL = j > 0 && Nc[j - 1] == N, sameR = j < nx - 1 && Nc[j + 1] == N;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n3; k += (size_t)gridDim.x * blockDim.x) {
    const double v1 = (int(k / ((size_t)N * N)) - N / 2) * h;
    const double c = v[o + k];
    double tv;
    if (v1 > 0) {
      const double left = j == 0 ? gs * gL[k] : (sameL ? v[off[j - 1] + k] : nb[o + k]);
      tv = v1 * (c - left) / dx;
    } else {
      const double right = j == nx - 1 ? gs * gR[k] : (sameR ? v[off[j + 1] + k] : nb[len + o + k]);
      tv = v1 * (right - c) / dx;
    }
    double r = cT * tv + cV * c;
    if (y) r += cY * y[o + k];
    out[o + k] = r;
  }
}

// per-cell sum of squares (for the weighted residual norm)
__global__ void __launch_bounds__(256) k_cell_sumsq(const double* __restrict__ r, const int* __restrict__ Nc,
                                                    const size_t* __restrict__ off, double* __restrict__ out) {
  __shared__ double sh[8];
  const int j = blockIdx.x, N = Nc[j], t = threadIdx.x;
  const size_t n3 = (size_t)N * N * N;
  double a = 0;
  for (size_t k = t; k < n3; k += 256) {
    const double x = r[off[j] + k];
    a += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((t & 31) == 0) sh[t >> 5] = a;
  __syncthreads();
  if (t == 0) {
    double v = 0;
    for (int i = 0; i < 8; ++i) v += sh[i];
    out[j] = v;
  }
}

// ------------------------------------------------------------ host helpers
std::vector<double> resample_matrix(int na, int nb, double L) {
  const long double pi = 3.14159265358979323846264338327950288L;
  const int K = std::min(na, nb) / 2;
  const long double c = nb > na ? 1.0L : 2.0L;
  const long double ha = 2.0L * L / na, hb = 2.0L * L / nb;
  std::vector<double> R((size_t)nb * na);
  for (int b = 0; b < nb; ++b) {
    const long double vb = (b - nb / 2) * hb;
    for (int a = 0; a < na; ++a) {
      const long double va = (a - na / 2) * ha;
      long double s = 1.0L;  // k = 0
      for (int k = 1; k < K; ++k) s += 2.0L * cosl(pi * k * (vb - va) / L);
      s += c * cosl(pi * K * va / L) * cosl(pi * K * vb / L);
      R[(size_t)b * na + a] = (double)(s / na);
    }
  }
  return R;
}

lbo_status upload_jobs(JobList& jl) {
  if (jl.host.empty()) return LBO_OK;
  cudaError_t e = cudaMalloc(&jl.dev, sizeof(RJob) * jl.host.size());
  if (e == cudaSuccess) e = cudaMemcpy(jl.dev, jl.host.data(), sizeof(RJob) * jl.host.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "mixed job list");
}

template <typename TC>
void run_jobs(lbo_solver* S, const JobList& jl, const double* src, double* dst) {
  MixedState* M = mstate(S);
  if (jl.host.empty()) return;
  const TC* mats;
  if constexpr (sizeof(TC) == 8) mats = M->mats64;
  else mats = M->mats32;
  LBO_LAUNCH(S->plan, "mixed_resample", S->plan->stream, k_resample_jobs<TC>, (int)jl.host.size(), RT, 0,
             jl.dev, src, dst, mats, M->tmp, (size_t)M->nmax * M->nmax * M->nmax);
}

// out (len layout) = plan(group) applied to v (len layout), per N group:
// L about the cells' local Maxwellians, or Q (residual plans if `residual`)
enum GroupOp { OP_LINEARIZED, OP_QUADRATIC };

lbo_status per_group(lbo_solver* S, GroupOp op, const double* v, double* out, bool residual) {
  MixedState* M = mstate(S);
  cudaStream_t s = S->plan->stream;
  for (Group& G : M->groups) {
    const int count = (int)G.cells.size();
    const size_t n3 = (size_t)G.N * G.N * G.N;
    const int bx = (int)std::min<size_t>(64, (n3 + 255) / 256);
    LBO_LAUNCH(S->plan, "mixed_gather", s, k_gather, dim3(bx, count), 256, 0, v, G.in, G.d_cells, M->d_off, n3, 1);
    lbo_plan* p = (residual && G.rplan) ? G.rplan : G.plan;
    p->stream = s;
    lbo_status st;
    if (op == OP_LINEARIZED) {
      LBO_LAUNCH(S->plan, "mixed_gather_params", s, k_gather_params, (5 * count + 255) / 256, 256, 0, S->params,
                 G.params, G.d_cells, count);
      st = lbo_apply_linearized(p, G.params, G.in, G.out, count);
    } else {
      st = lbo_apply_quadratic(p, G.in, G.out, count);
    }
    if (st != LBO_OK) return st;
    LBO_LAUNCH(S->plan, "mixed_scatter", s, k_gather, dim3(bx, count), 256, 0, G.out, out, G.d_cells, M->d_off, n3,
               0);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "mixed collisions");
}

void transport(lbo_solver* S, const double* v, const double* y, double* out, double cY, double gs, double cV,
               bool fp64) {
  MixedState* M = mstate(S);
  if (fp64) run_jobs<double>(S, M->transport, v, M->nb2);
  else run_jobs<float>(S, M->transport, v, M->nb2);
  const int bx = (int)std::min<size_t>(64, ((size_t)M->nmax * M->nmax * M->nmax + 255) / 256);
  LBO_LAUNCH(S->plan, "mixed_transport", S->plan->stream, k_mixed_transport, dim3(bx, M->nx), 256, 0, v, y,
             M->nb2, M->len, M->gL, M->gR, out, M->d_N, M->d_off, M->nx, M->L, S->dx, 1.0, cY, gs, cV);
}

}  // namespace

// ------------------------------------------------------------ solver hooks
void mixed_moments(lbo_solver* S, const double* f, double* params, double* nu) {
  MixedState* M = mstate(S);
  LBO_LAUNCH(S->plan, "mixed_moments", S->plan->stream, k_mixed_moments, M->nx, 256, 0, f, M->d_N, M->d_off, M->L,
             params, nu);
}

lbo_status mixed_residual(lbo_solver* S, const double* f, double* out, double* nrm) {
  MixedState* M = mstate(S);
  lbo_status st = per_group(S, OP_QUADRATIC, f, S->Qf, true);
  if (st != LBO_OK) return st;
  transport(S, f, S->Qf, out, -1.0 / S->pb.kn, 1.0, 0.0, true);
  if (nrm) {
    // sqrt(dx sum_j h_j^3 sum r_j^2), cell by cell
    LBO_LAUNCH(S->plan, "mixed_sumsq", S->plan->stream, k_cell_sumsq, M->nx, 256, 0, out, M->d_N, M->d_off, S->part);
    std::vector<double> h(M->nx);
    cudaMemcpyAsync(h.data(), S->part, sizeof(double) * M->nx, cudaMemcpyDeviceToHost, S->plan->stream);
    cudaError_t e = cudaStreamSynchronize(S->plan->stream);
    if (e != cudaSuccess) return cuda_fail(e, "mixed residual norm");
    double acc = 0;
    for (int j = 0; j < M->nx; ++j) {
      const double hj = 2.0 * M->L / M->Nc[j];
      acc += hj * hj * hj * h[j];
    }
    *nrm = std::sqrt(S->dx * acc);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "mixed residual");
}

// out = T v - C v / Kn + shift v; C = L about the local Maxwellians, or the
// exact J_Q v = (Q(f + s v) - Q(f - s v)) / (2 s)
lbo_status mixed_apply_op(lbo_solver* S, const double* v, double* out) {
  lbo_status st;
  if (S->pb.jacobian == 1) {
    const double vn = solver_norm2(S, v, &st);
    if (st != LBO_OK) return st;
    const double sc = (vn > 0 && S->fnorm > 0) ? S->fnorm / vn : 1.0;
    cudaStream_t s = S->plan->stream;
    for (int side = 0; side < 2; ++side) {
      double* x = side == 0 ? S->ja : S->jb;
      cudaMemcpyAsync(x, S->fcur, sizeof(double) * S->len, cudaMemcpyDeviceToDevice, s);
      solver_axpby(S, x, v, side == 0 ? sc : -sc, 1.0);
    }
    st = per_group(S, OP_QUADRATIC, S->ja, S->Lv, false);
    if (st == LBO_OK) st = per_group(S, OP_QUADRATIC, S->jb, S->ja, false);
    if (st != LBO_OK) return st;
    solver_axpby(S, S->Lv, S->ja, -0.5 / sc, 0.5 / sc);
  } else {
    st = per_group(S, OP_LINEARIZED, v, S->Lv, false);
    if (st != LBO_OK) return st;
  }
  // neighbours resampled in the operator plan's precision
  transport(S, v, S->Lv, out, -1.0 / S->pb.kn, 0.0, S->shift, S->plan->precision != LBO_PREC_FP32);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "mixed operator");
}

// the upwind sweep of Eq. (5.7) on the finest grid: resample, sweep, back
lbo_status mixed_sweep(lbo_solver* S, const double* v, double* z) {
  MixedState* M = mstate(S);
  run_jobs<float>(S, M->to_max, v, M->sweep_in);
  lbo_status st = solver_sweep_uniform(S, M->sweep_in, M->sweep_out, M->nmax, 2.0 * M->L / M->nmax);
  if (st != LBO_OK) return st;
  run_jobs<float>(S, M->from_max, M->sweep_out, z);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "mixed sweep");
}

lbo_status mixed_set_residual_plan(lbo_solver* S, lbo_plan* plan) {
  MixedState* M = mstate(S);
  if (!plan) {
    for (Group& G : M->groups) G.rplan = nullptr;
    return LBO_OK;
  }
  for (Group& G : M->groups)
    if (G.N == plan->N && plan->L == M->L) {
      G.rplan = plan;
      return LBO_OK;
    }
  return LBO_EINVAL;
}

void free_mixed(lbo_solver* S) {
  MixedState* M = mstate(S);
  if (!M) return;
  for (Group& G : M->groups) {
    cudaFree(G.d_cells);
    cudaFree(G.in);
    cudaFree(G.out);
    cudaFree(G.params);
  }
  void* ptrs[] = {M->d_N, M->d_off, M->nb2, M->gL, M->gR, M->mats64, M->mats32, M->tmp, M->sweep_in,
                  M->sweep_out, M->transport.dev, M->to_max.dev, M->from_max.dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete M;
  S->mixed = nullptr;
}

// Builds the mixed state on a solver whose uniform buffers are sized for
// len = sum_j N_j^3 (see lbo_solver_create_mixed).
lbo_status mixed_setup(lbo_solver* S, lbo_plan* const* plans, int nplans, const int* cell_plan) {
  auto* M = new MixedState();
  S->mixed = M;
  M->nx = S->nx;
  M->L = plans[0]->L;
  M->Nc.resize(M->nx);
  M->off.resize(M->nx);
  size_t o = 0;
  for (int j = 0; j < M->nx; ++j) {
    M->Nc[j] = plans[cell_plan[j]]->N;
    M->off[j] = o;
    o += (size_t)M->Nc[j] * M->Nc[j] * M->Nc[j];
    M->nmax = std::max(M->nmax, M->Nc[j]);
  }
  M->len = o;
  cudaError_t e = cudaSuccess;
  auto dalloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  dalloc((void**)&M->d_N, sizeof(int) * M->nx);
  dalloc((void**)&M->d_off, sizeof(size_t) * M->nx);
  if (e == cudaSuccess) e = cudaMemcpy(M->d_N, M->Nc.data(), sizeof(int) * M->nx, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(M->d_off, M->off.data(), sizeof(size_t) * M->nx, cudaMemcpyHostToDevice);
  // groups
  for (int p = 0; p < nplans; ++p) {
    Group G;
    G.plan = plans[p];
    G.N = plans[p]->N;
    for (int j = 0; j < M->nx; ++j)
      if (cell_plan[j] == p) G.cells.push_back(j);
    if (G.cells.empty()) continue;
    const size_t n3 = (size_t)G.N * G.N * G.N, cnt = G.cells.size();
    dalloc((void**)&G.d_cells, sizeof(int) * cnt);
    dalloc((void**)&G.in, sizeof(double) * cnt * n3);
    dalloc((void**)&G.out, sizeof(double) * cnt * n3);
    dalloc((void**)&G.params, sizeof(double) * cnt * 5);
    if (e == cudaSuccess) e = cudaMemcpy(G.d_cells, G.cells.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice);
    M->groups.push_back(G);
  }
  // resampling matrices for every ordered pair in use (the finest grid included)
  std::map<std::pair<int, int>, int> mat_of;
  std::vector<double> mats;
  auto mat = [&](int na, int nb) {
    if (na == nb) return 0;
    auto key = std::make_pair(na, nb);
    auto it = mat_of.find(key);
    if (it != mat_of.end()) return it->second;
    const int at = (int)mats.size();
    std::vector<double> R = resample_matrix(na, nb, M->L);
    mats.insert(mats.end(), R.begin(), R.end());
    mat_of[key] = at;
    return at;
  };
  const size_t cube = (size_t)M->nmax * M->nmax * M->nmax;
  size_t njobs = 0;  // jobs that resample (copies need no scratch)
  auto job = [&](JobList& jl, size_t src, size_t dst, int na, int nb) {
    jl.host.push_back(RJob{src, dst, na == nb ? 0 : 2 * cube * njobs++, na, nb, mat(na, nb)});
  };
  for (int j = 0; j < M->nx; ++j) {
    if (j > 0 && M->Nc[j - 1] != M->Nc[j]) job(M->transport, M->off[j - 1], M->off[j], M->Nc[j - 1], M->Nc[j]);
    if (j < M->nx - 1 && M->Nc[j + 1] != M->Nc[j])
      job(M->transport, M->off[j + 1], M->len + M->off[j], M->Nc[j + 1], M->Nc[j]);
  }
  const size_t nm3 = (size_t)M->nmax * M->nmax * M->nmax;
  for (int j = 0; j < M->nx; ++j) job(M->to_max, M->off[j], j * nm3, M->Nc[j], M->nmax);
  for (int j = 0; j < M->nx; ++j) job(M->from_max, j * nm3, M->off[j], M->nmax, M->Nc[j]);
  std::vector<float> mats32(mats.begin(), mats.end());
  if (mats.empty()) {
    mats.push_back(0.0);
    mats32.push_back(0.0f);
  }
  dalloc((void**)&M->mats64, sizeof(double) * mats.size());
  dalloc((void**)&M->mats32, sizeof(float) * mats32.size());
  if (e == cudaSuccess) e = cudaMemcpy(M->mats64, mats.data(), sizeof(double) * mats.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(M->mats32, mats32.data(), sizeof(float) * mats32.size(), cudaMemcpyHostToDevice);
  dalloc((void**)&M->tmp, sizeof(double) * 2 * cube * std::max<size_t>(njobs, 1));
  dalloc((void**)&M->nb2, sizeof(double) * 2 * M->len);
  dalloc((void**)&M->sweep_in, sizeof(double) * M->nx * nm3);
  dalloc((void**)&M->sweep_out, sizeof(double) * M->nx * nm3);
  // inflow ghosts on the boundary cells' grids
  for (int side = 0; side < 2; ++side) {
    const int N = M->Nc[side == 0 ? 0 : M->nx - 1];
    const double* in = side == 0 ? S->pb.inflow_left : S->pb.inflow_right;
    const double h = 2.0 * M->L / N;
    std::vector<double> gh((size_t)N * N * N);
    for (size_t k = 0; k < gh.size(); ++k) {
      const int i1 = (int)(k / ((size_t)N * N)), i2 = (int)((k / N) % N), i3 = (int)(k % N);
      const double d1 = (i1 - N / 2) * h - in[1], d2 = (i2 - N / 2) * h - in[2], d3 = (i3 - N / 2) * h - in[3];
      gh[k] = in[0] * std::pow(2.0 * 3.141592653589793 * in[4], -1.5) *
              std::exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * in[4]));
    }
    double** dst = side == 0 ? &M->gL : &M->gR;
    dalloc((void**)dst, sizeof(double) * gh.size());
    if (e == cudaSuccess) e = cudaMemcpy(*dst, gh.data(), sizeof(double) * gh.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(e, "mixed set-up");
  lbo_status st = upload_jobs(M->transport);
  if (st == LBO_OK) st = upload_jobs(M->to_max);
  if (st == LBO_OK) st = upload_jobs(M->from_max);
  return st;
}

size_t mixed_state_length(const lbo_plan* const* plans, int nx, const int* cell_plan) {
  size_t o = 0;
  for (int j = 0; j < nx; ++j) o += (size_t)plans[cell_plan[j]]->N * plans[cell_plan[j]]->N * plans[cell_plan[j]]->N;
  return o;
}

}  // namespace lbo

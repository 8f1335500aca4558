// Two-level preconditioner for the slab's linear step: the upwind sweep of
// the source iteration (Eq. (5.7)) followed by a coarse correction on the
// low moments of every cell: the five collision invariants, optionally
// widened by the traceless stress and the heat flux (Grad's 13 moments).
//
// The sweep leaves the conserved moments almost untouched when Kn is small:
// collisions do not damp them.  The five invariants alone carry only the
// Euler fluxes; stress and heat flux add the viscous and conductive coupling.  This is the synthetic acceleration that Sec. 5.2
// points to for small Kn, in Galerkin form:
//
//   P_j,b(v) = M_j(v) psi_b(xi),  xi = (v - u_j) / sqrt(theta_j),
//   psi = {1, xi_1, xi_2, xi_3, |xi|^2/2 - 3/2}                  (5), then
//         xi_1 xi_2, xi_1 xi_3, xi_2 xi_3, xi_1^2 - |xi|^2/3,
//         xi_2^2 - |xi|^2/3, xi_i (|xi|^2/2 - 5/2)               (13),
//   (W^T r)_j,a = h^3 sum_v psi_a(xi) r_j(v)      (cell-local moments),
//   A_c = W^T A' P   (5 nx x 5 nx, assembled from A' itself),
//   z = S r;  z += P A_c^{-1} W^T (r - A' z).
//
// A' couples only neighbouring cells, apart from the rank-one mass border
// e m(g) between two walls.  So A_c is block tridiagonal with nb x nb blocks
// plus a rank-one term.  It is assembled from 3 nb applications of A' to
// basis vectors coloured mod 3 (no two cells of one colour share a
// neighbour), and factored on the host by banded LU with partial pivoting.
// The rank-one border becomes one extra row and column (an arrow).
//
// coarse_operator = 1 replaces A' by its transport, border and shift parts
// in both the assembly and the residual r - A' z.  For the five collision
// invariants this drops only what the discrete collision operator fails to
// conserve (W^T L P = 0 and W^T J_Q P = 0 in exact arithmetic), and it saves
// the collision-operator application that the Galerkin form spends per
// Krylov iteration: the low-order moment equation of synthetic
// acceleration.
#include <cmath>
#include <cstring>
#include <vector>

#include "lbo_internal.h"

namespace lbo {
namespace {

constexpr int CT = 256;   // threads per cell block

struct CoarseState {
  int nx = 0, nb = 5, nc = 0;
  int kl = 9, ku = 9, bw = 28;  // bandwidths 2 nb - 1; row window [r - kl, r + kl + ku]
  double* d_vec = nullptr;   // basis vector / residual scratch (len)
  double* d_out = nullptr;   // A' applied to it (len)
  double* d_mom = nullptr;   // nb nx moments / coefficients
  double* h_mom = nullptr;   // pinned copy
  std::vector<double> ab;    // LU factors, nc rows x BW window
  std::vector<double> pc, qr;  // arrow column / row (factored in place)
  std::vector<int> piv;
  double d = -1.0;           // arrow corner
  double t00 = 0, t01 = 0, t10 = 0, t11 = 0;  // trailing 2 x 2 system
  bool valid = false;
};

__device__ __forceinline__ void xi_of(int k, int N, double h, const double* p, double* x) {
  const int i1 = k / (N * N), i2 = (k / N) % N, i3 = k % N;
  const double s = rsqrt(p[4]);
  x[0] = ((i1 - N / 2) * h - p[1]) * s;
  x[1] = ((i2 - N / 2) * h - p[2]) * s;
  x[2] = ((i3 - N / 2) * h - p[3]) * s;
}

template <int NB>
__device__ __forceinline__ void psi_of(const double* x, double* psi) {
  const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  psi[0] = 1.0;
  psi[1] = x[0];
  psi[2] = x[1];
  psi[3] = x[2];
  psi[4] = 0.5 * r2 - 1.5;
  if (NB == 13) {
    psi[5] = x[0] * x[1];
    psi[6] = x[0] * x[2];
    psi[7] = x[1] * x[2];
    psi[8] = x[0] * x[0] - r2 / 3.0;
    psi[9] = x[1] * x[1] - r2 / 3.0;
    const double q = 0.5 * r2 - 2.5;
    psi[10] = x[0] * q;
    psi[11] = x[1] * q;
    psi[12] = x[2] * q;
  }
}

// out[NB j + a] = h^3 sum_v psi_a(xi_j(v)) v_j(v); grid nx blocks
template <int NB>
__global__ void __launch_bounds__(CT) k_coarse_restrict(const double* __restrict__ v,
                                                        const double* __restrict__ params, double* __restrict__ out,
                                                        int N, double h) {
  __shared__ double sh[NB][CT / 32];
  const int j = blockIdx.x, n3 = N * N * N;
  const double* p = params + 5 * j;
  const double* vj = v + (size_t)j * n3;
  double acc[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) acc[a] = 0.0;
  for (int k = threadIdx.x; k < n3; k += CT) {
    double x[3], psi[NB];
    xi_of(k, N, h, p, x);
    psi_of<NB>(x, psi);
    const double val = vj[k];
#pragma unroll
    for (int a = 0; a < NB; ++a) acc[a] += psi[a] * val;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    double t = acc[a];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh[a][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    double t = 0;
    for (int i = 0; i < CT / 32; ++i) t += sh[threadIdx.x][i];
    out[NB * j + threadIdx.x] = h * h * h * t;
  }
}

// colour >= 0: z_j = (j mod 3 == colour) ? M_j psi_b : 0   (assembly basis)
// colour <  0: z_j += M_j sum_b c[NB j + b] psi_b           (prolongation)
template <int NB>
__global__ void k_coarse_prolong(double* __restrict__ z, const double* __restrict__ params,
                                 const double* __restrict__ c, int N, double h, int colour, int b) {
  const int j = blockIdx.y, n3 = N * N * N;
  const double* p = params + 5 * j;
  double* zj = z + (size_t)j * n3;
  const bool on = colour < 0 || j % 3 == colour;
  const double norm = p[0] * pow(2.0 * 3.141592653589793 * p[4], -1.5);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += gridDim.x * blockDim.x) {
    if (!on) {
      zj[k] = 0.0;
      continue;
    }
    double x[3], psi[NB];
    xi_of(k, N, h, p, x);
    psi_of<NB>(x, psi);
    const double m = norm * exp(-0.5 * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]));
    if (colour >= 0) {
      zj[k] = m * psi[b];
    } else {
      const double* cj = c + NB * j;
      double acc = 0.0;
#pragma unroll
      for (int a = 0; a < NB; ++a) acc += cj[a] * psi[a];
      zj[k] += m * acc;
    }
  }
}

CoarseState* state(lbo_solver* S) { return static_cast<CoarseState*>(S->coarse); }

double& at(CoarseState* C, int r, int c) { return C->ab[(size_t)r * C->bw + (c - r + C->kl)]; }

// Banded LU with partial pivoting of the arrow matrix [B p; q^T d], the band
// columns 0..nc-2 first, then the trailing 2 x 2 block (last band unknown
// and the border multiplier) with its own pivoting.
bool factor(CoarseState* C) {
  const int n = C->nc;
  C->piv.assign(n, 0);
  double scale = 0;
  for (double v : C->ab) scale = std::fmax(scale, std::fabs(v));
  const double tiny = 1e-14 * (scale > 0 ? scale : 1.0);
  const int KL = C->kl, KU = C->ku;
  for (int k = 0; k < n - 1; ++k) {
    const int last = std::min(n - 1, k + KL);
    int p = k;
    double best = std::fabs(at(C, k, k));
    for (int r = k + 1; r <= last; ++r)
      if (std::fabs(at(C, r, k)) > best) best = std::fabs(at(C, r, k)), p = r;
    if (!(best > tiny)) return false;
    C->piv[k] = p;
    const int cend = std::min(n - 1, k + KL + KU);
    if (p != k) {
      for (int c = k; c <= cend; ++c) std::swap(at(C, k, c), at(C, p, c));
      std::swap(C->pc[k], C->pc[p]);
    }
    const double dk = at(C, k, k);
    for (int r = k + 1; r <= last; ++r) {
      const double l = at(C, r, k) / dk;
      at(C, r, k) = l;
      if (l == 0.0) continue;
      for (int c = k + 1; c <= cend; ++c) at(C, r, c) -= l * at(C, k, c);
      C->pc[r] -= l * C->pc[k];
    }
    const double l = C->qr[k] / dk;
    C->qr[k] = l;
    for (int c = k + 1; c <= cend; ++c) C->qr[c] -= l * at(C, k, c);
    C->d -= l * C->pc[k];
  }
  C->piv[n - 1] = n - 1;
  C->t00 = at(C, n - 1, n - 1);
  C->t01 = C->pc[n - 1];
  C->t10 = C->qr[n - 1];
  C->t11 = C->d;
  const double det = C->t00 * C->t11 - C->t01 * C->t10;
  const double sz = std::fabs(C->t00 * C->t11) + std::fabs(C->t01 * C->t10);
  return std::isfinite(det) && std::fabs(det) > 1e-14 * (sz > 0 ? sz : 1.0);
}

// Solve [B p; q^T d] [x; s] = [b; 0] in place (b -> x).
void solve(CoarseState* C, double* b) {
  const int n = C->nc, KL = C->kl, KU = C->ku;
  double bn = 0.0;
  for (int k = 0; k < n - 1; ++k) {
    if (C->piv[k] != k) std::swap(b[k], b[C->piv[k]]);
    const int last = std::min(n - 1, k + KL);
    for (int r = k + 1; r <= last; ++r) b[r] -= at(C, r, k) * b[k];
    bn -= C->qr[k] * b[k];
  }
  const double det = C->t00 * C->t11 - C->t01 * C->t10;
  const double xl = (b[n - 1] * C->t11 - C->t01 * bn) / det;
  const double s = (C->t00 * bn - C->t10 * b[n - 1]) / det;
  b[n - 1] = xl;
  for (int k = n - 2; k >= 0; --k) {
    double acc = b[k] - C->pc[k] * s;
    const int cend = std::min(n - 1, k + KL + KU);
    for (int c = k + 1; c <= cend; ++c) acc -= at(C, k, c) * b[c];
    b[k] = acc / at(C, k, k);
  }
}

lbo_status ensure(lbo_solver* S) {
  if (S->coarse) return LBO_OK;
  auto* C = new CoarseState();
  C->nx = S->nx;
  C->nb = S->pb.coarse_moments == 13 ? 13 : 5;
  C->nc = C->nb * S->nx;
  C->kl = C->ku = 2 * C->nb - 1;
  C->bw = 2 * C->kl + C->ku + 1;
  cudaError_t e = cudaMalloc(&C->d_vec, sizeof(double) * S->len);
  if (e == cudaSuccess) e = cudaMalloc(&C->d_out, sizeof(double) * S->len);
  if (e == cudaSuccess) e = cudaMalloc(&C->d_mom, sizeof(double) * C->nc);
  if (e == cudaSuccess) e = cudaMallocHost(&C->h_mom, sizeof(double) * C->nc);
  S->coarse = C;
  if (e != cudaSuccess) return cuda_fail(e, "coarse workspace");
  return LBO_OK;
}

lbo_status restrict_to_host(lbo_solver* S, const double* v) {
  CoarseState* C = state(S);
  cudaStream_t s = S->plan->stream;
  if (C->nb == 13)
    LBO_LAUNCH(S->plan, "coarse_restrict", s, k_coarse_restrict<13>, S->nx, CT, 0, v, S->params, C->d_mom, S->N,
               S->h);
  else
    LBO_LAUNCH(S->plan, "coarse_restrict", s, k_coarse_restrict<5>, S->nx, CT, 0, v, S->params, C->d_mom, S->N,
               S->h);
  cudaMemcpyAsync(C->h_mom, C->d_mom, sizeof(double) * C->nc, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "coarse restriction");
}

dim3 prolong_grid(const lbo_solver* S) {
  const int per = (int)((S->n3 + 255) / 256);
  return dim3(per < 64 ? per : 64, S->nx);
}

void prolong(lbo_solver* S, double* z, const double* c, int colour, int b) {
  CoarseState* C = state(S);
  if (C->nb == 13)
    LBO_LAUNCH(S->plan, colour >= 0 ? "coarse_basis" : "coarse_prolong", S->plan->stream, k_coarse_prolong<13>,
               prolong_grid(S), 256, 0, z, S->params, c, S->N, S->h, colour, b);
  else
    LBO_LAUNCH(S->plan, colour >= 0 ? "coarse_basis" : "coarse_prolong", S->plan->stream, k_coarse_prolong<5>,
               prolong_grid(S), 256, 0, z, S->params, c, S->N, S->h, colour, b);
}

}  // namespace

// Assemble and factor A_c = W^T A' P about the current cell parameters.
lbo_status coarse_assemble(lbo_solver* S, bool border) {
  lbo_status st = ensure(S);
  if (st != LBO_OK) return st;
  CoarseState* C = state(S);
  const int nx = S->nx, nc = C->nc, nb = C->nb;
  C->ab.assign((size_t)nc * C->bw, 0.0);
  C->pc.assign(nc, 0.0);
  C->qr.assign(nc, 0.0);
  C->d = -1.0;
  C->valid = false;
  for (int colour = 0; colour < 3; ++colour) {
    for (int b = 0; b < nb; ++b) {
      prolong(S, C->d_vec, nullptr, colour, b);
      if (border) {
        // q_(j,b) = m(P_(j,b)) = dx h^3 sum_v P_(j,b): the a = 0 moment
        st = restrict_to_host(S, C->d_vec);
        if (st != LBO_OK) return st;
        for (int j = colour; j < nx; j += 3) C->qr[nb * j + b] = S->dx * C->h_mom[nb * j];
      }
      st = solver_apply_op(S, C->d_vec, C->d_out, false, S->pb.coarse_operator != 1);
      if (st != LBO_OK) return st;
      st = restrict_to_host(S, C->d_out);
      if (st != LBO_OK) return st;
      for (int i = 0; i < nx; ++i) {
        int j = i - 1;
        while (j < 0 || (j % 3) != colour) ++j;  // the cell of this colour among i-1, i, i+1
        if (j > i + 1 || j >= nx) continue;
        for (int a = 0; a < nb; ++a) at(C, nb * i + a, nb * j + b) = C->h_mom[nb * i + a];
      }
    }
  }
  if (border) {
    // p = W^T e with e = f / m(f), the border's direction
    st = restrict_to_host(S, S->evec);
    if (st != LBO_OK) return st;
    for (int r = 0; r < nc; ++r) C->pc[r] = C->h_mom[r];
  }
  C->valid = factor(C);
  return LBO_OK;
}

bool coarse_valid(const lbo_solver* S) {
  return S->coarse && static_cast<const CoarseState*>(S->coarse)->valid;
}

// z holds the sweep of v on entry; adds P A_c^{-1} W^T (v - A' z).
lbo_status coarse_correct(lbo_solver* S, const double* v, double* z) {
  CoarseState* C = state(S);
  if (!C || !C->valid) return LBO_OK;
  cudaStream_t s = S->plan->stream;
  lbo_status st = solver_apply_op(S, z, C->d_out, true, S->pb.coarse_operator != 1);
  if (st != LBO_OK) return st;
  solver_axpby(S, C->d_out, v, 1.0, -1.0);  // v - A' z
  st = restrict_to_host(S, C->d_out);
  if (st != LBO_OK) return st;
  solve(C, C->h_mom);
  for (int r = 0; r < C->nc; ++r)
    if (!std::isfinite(C->h_mom[r])) return LBO_ENAN;
  cudaMemcpyAsync(C->d_mom, C->h_mom, sizeof(double) * C->nc, cudaMemcpyHostToDevice, s);
  prolong(S, z, C->d_mom, -1, 0);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "coarse correction");
}

void free_coarse(lbo_solver* S) {
  CoarseState* C = state(S);
  if (!C) return;
  cudaFree(C->d_vec);
  cudaFree(C->d_out);
  cudaFree(C->d_mom);
  cudaFreeHost(C->h_mom);
  delete C;
  S->coarse = nullptr;
}

}  // namespace lbo

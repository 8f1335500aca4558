// Learned preconditioner: a two-layer 1-D convolutional network over the
// cells of a slab that predicts the macroscopic part of the error left by
// the upwind sweep (the synthetic acceleration the paper points to for small
// Kn, Sec. 5.2; the network itself has no counterpart in the paper).
//
//   features of a vector v (per cell j): x_j = [m(r_j), m(s_j)], s = sweep(v),
//     r = v - A_T s the part of v the sweep leaves unexplained, A_T the
//     operator without its collision term (upwind transport, wall ghosts,
//     mass border, shift): for the collision invariants W^T A = W^T A_T up
//     to the discrete operator's conservation, so the five low moments of r
//     drive the macroscopic error of s exactly as in synthetic acceleration;
//     m(y)_a = h^3 sum_v phi_a(v) y(v), phi = 13 moments (below);
//   network: h1 = tanh(b1 + W1 * x), y = b2 + W2 * h1 (width-5 convolutions
//     over cells, zero padding, H hidden channels, 5 outputs);
//   preconditioner: z = s + sum_a c_{j,a} phi_a(v) M_j(v),
//     c = sigma cs_out (.) y((x / sigma) / cs_in), sigma = RMS of m(s) over
//     the slab (so that z is positively homogeneous in v).
// Training pairs are (A z_k, z_k) from the solver's own FGMRES iterations:
// the target c_j solves G_j c_j = m(z_j) - m(s_j), G_j the 5x5 moment matrix
// of phi_a phi_b M_j.  Training: full-batch Adam on the mean squared error,
// FP32 weights, hand-written forward/backward kernels.  FGMRES keeps the
// exact operator as the measure of convergence, so a poor network costs iterations only.
#include <cmath>
#include <cstring>
#include <vector>

#include "lbo_internal.h"

namespace lbo {

struct NetState {
  int hidden = 0;
  int max_pairs = 0, pairs = 0;
  bool collecting = false;
  float* store_x = nullptr;  // [max_pairs][nx][26] raw features (13 moments of v and of its sweep)
  float* store_t = nullptr;  // [max_pairs][nx][5] raw targets
  float* theta = nullptr;    // device parameters
  float scales[31] = {};  // cs_in[26], cs_out[5]
  float* feat = nullptr;     // [nx][26] features of the vector being preconditioned
  float* corr = nullptr;     // [nx][5]
  double* r = nullptr;       // v - A_T s of the vector being preconditioned or recorded
  float* dev_sc = nullptr;   // scales on the device, then sigma of the current vector
  bool trained = false;
};

namespace {

constexpr int NMOM = 13, CIN = 2 * NMOM, COUT = 5, KW = 5;

int param_count(int H) { return H * CIN * KW + H + COUT * H * KW + COUT; }
// hidden = 0 selects the global linear form, whose size depends on nx
size_t param_count_nx(int H, int nx) {
  return H > 0 ? (size_t)param_count(H) : (size_t)COUT * CIN * (2 * nx - 1) + COUT;
}

__device__ __forceinline__ double bsum(double v, double* sh) {
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

// phi_0..4 = 1, v1, v2, v3, |v|^2 (collision invariants; the lift basis);
// phi_5..12 = v1 v2, v1 v3, v2 v3, v1^2 - v2^2, v2^2 - v3^2, v1|v|^2, v2|v|^2,
// v3|v|^2 (stress and heat-flux moments, input features only)
__device__ __forceinline__ void phis(int k, int N, double h, double* ph) {
  const int i1 = k / (N * N), i2 = (k / N) % N, i3 = k % N;
  const double v1 = (i1 - N / 2) * h, v2 = (i2 - N / 2) * h, v3 = (i3 - N / 2) * h;
  const double q = v1 * v1 + v2 * v2 + v3 * v3;
  ph[0] = 1.0;
  ph[1] = v1;
  ph[2] = v2;
  ph[3] = v3;
  ph[4] = q;
  ph[5] = v1 * v2;
  ph[6] = v1 * v3;
  ph[7] = v2 * v3;
  ph[8] = v1 * v1 - v2 * v2;
  ph[9] = v2 * v2 - v3 * v3;
  ph[10] = v1 * q;
  ph[11] = v2 * q;
  ph[12] = v3 * q;
}

// One block per cell: the 13 moments of v and of s (features), and for
// training pairs also the target c_j from z and the cell Maxwellian.
__global__ void __launch_bounds__(256) k_cell_features(const double* __restrict__ v, const double* __restrict__ s,
                                                       const double* __restrict__ z, const double* __restrict__ params,
                                                       int N, double h, float* __restrict__ xout,
                                                       float* __restrict__ tout) {
  constexpr int NA = 2 * NMOM + 5 + 15;
  __shared__ double sh[32];
  __shared__ double res[NA];
  const int j = blockIdx.x;
  const int n3 = N * N * N;
  const double* vj = v + (size_t)j * n3;
  const double* sj = s + (size_t)j * n3;
  const double* zj = z ? z + (size_t)j * n3 : nullptr;
  const double rho = params[5 * j], u1 = params[5 * j + 1], u2 = params[5 * j + 2], u3 = params[5 * j + 3],
               th = params[5 * j + 4];
  const double pref = rho * pow(2.0 * 3.141592653589793 * th, -1.5);
  double acc[NA];
  for (int i = 0; i < NA; ++i) acc[i] = 0.0;
  for (int k = threadIdx.x; k < n3; k += blockDim.x) {
    double ph[NMOM];
    phis(k, N, h, ph);
    const double a = vj[k], b = sj[k];
    for (int q = 0; q < NMOM; ++q) {
      acc[q] += ph[q] * a;
      acc[NMOM + q] += ph[q] * b;
    }
    if (zj) {
      const double c = zj[k];
      for (int q = 0; q < 5; ++q) acc[2 * NMOM + q] += ph[q] * c;
      const double d1 = ph[1] - u1, d2 = ph[2] - u2, d3 = ph[3] - u3;
      const double M = pref * exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * th));
      int idx = 2 * NMOM + 5;
      for (int p = 0; p < 5; ++p)
        for (int q = p; q < 5; ++q) acc[idx++] += ph[p] * ph[q] * M;
    }
  }
  const int nres = zj ? NA : 2 * NMOM;
  for (int i = 0; i < nres; ++i) {
    double r = bsum(acc[i], sh);
    if (threadIdx.x == 0) res[i] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double h3 = h * h * h;
    for (int q = 0; q < CIN; ++q) xout[j * CIN + q] = (float)(h3 * res[q]);
    if (zj) {
      double G[5][6];
      int idx = 2 * NMOM + 5;
      for (int p = 0; p < 5; ++p)
        for (int q = p; q < 5; ++q) {
          G[p][q] = G[q][p] = h3 * res[idx++];
        }
      for (int p = 0; p < 5; ++p) G[p][5] = h3 * (res[2 * NMOM + p] - res[NMOM + p]);
      for (int c = 0; c < 5; ++c) {  // Gaussian elimination with partial pivoting
        int piv = c;
        for (int r = c + 1; r < 5; ++r)
          if (fabs(G[r][c]) > fabs(G[piv][c])) piv = r;
        for (int q = 0; q < 6; ++q) {
          double tmp = G[c][q];
          G[c][q] = G[piv][q];
          G[piv][q] = tmp;
        }
        for (int r = 0; r < 5; ++r)
          if (r != c && G[c][c] != 0.0) {
            double f = G[r][c] / G[c][c];
            for (int q = c; q < 6; ++q) G[r][q] -= f * G[c][q];
          }
      }
      for (int p = 0; p < 5; ++p) tout[j * COUT + p] = G[p][p] != 0.0 ? (float)(G[p][5] / G[p][p]) : 0.f;
    }
  }
}

// ---------------------------------------------------------------- network
struct NetPtr {
  const float *W1, *b1, *W2, *b2;
};
__device__ __forceinline__ NetPtr net_ptr(const float* th, int H) {
  NetPtr n;
  n.W1 = th;
  n.b1 = n.W1 + H * CIN * KW;
  n.W2 = n.b1 + H;
  n.b2 = n.W2 + COUT * H * KW;
  return n;
}

// h1[p][j][o] = tanh(b1 + sum W1 x)
__global__ void k_fwd1(const float* __restrict__ th, int H, const float* __restrict__ x, int P, int nx,
                       float* __restrict__ h1) {
  const NetPtr n = net_ptr(th, H);
  const size_t total = (size_t)P * nx * H;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(t % H), j = (int)((t / H) % nx), p = (int)(t / ((size_t)H * nx));
    float acc = n.b1[o];
    for (int d = 0; d < KW; ++d) {
      const int jj = j + d - 2;
      if (jj < 0 || jj >= nx) continue;
      const float* xr = x + ((size_t)p * nx + jj) * CIN;
      for (int c = 0; c < CIN; ++c) acc += n.W1[(o * CIN + c) * KW + d] * xr[c];
    }
    h1[t] = tanhf(acc);
  }
}

// y = b2 + sum W2 h1; with targets: dy = 2 (y - t)/count and squared errors
__global__ void k_fwd2(const float* __restrict__ th, int H, const float* __restrict__ h1, int P, int nx,
                       const float* __restrict__ t, float* __restrict__ y, float* __restrict__ dy,
                       float* __restrict__ se) {
  const NetPtr n = net_ptr(th, H);
  const size_t total = (size_t)P * nx * COUT;
  const float inv = 1.0f / (float)total;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(q % COUT), j = (int)((q / COUT) % nx), p = (int)(q / ((size_t)COUT * nx));
    float acc = n.b2[a];
    for (int d = 0; d < KW; ++d) {
      const int jj = j + d - 2;
      if (jj < 0 || jj >= nx) continue;
      const float* hr = h1 + ((size_t)p * nx + jj) * H;
      for (int o = 0; o < H; ++o) acc += n.W2[(a * H + o) * KW + d] * hr[o];
    }
    if (y) y[q] = acc;
    if (t) {
      const float e = acc - t[q];
      dy[q] = 2.0f * e * inv;
      se[q] = e * e;
    }
  }
}

// dz1[p][j][o] = (1 - h1^2) sum_{a,d} W2[a][o][d] dy[p][j - d + 2][a]
__global__ void k_bwd1(const float* __restrict__ th, int H, const float* __restrict__ h1,
                       const float* __restrict__ dy, int P, int nx, float* __restrict__ dz1) {
  const NetPtr n = net_ptr(th, H);
  const size_t total = (size_t)P * nx * H;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int o = (int)(t % H), j = (int)((t / H) % nx), p = (int)(t / ((size_t)H * nx));
    float acc = 0.f;
    for (int d = 0; d < KW; ++d) {
      const int jy = j - d + 2;
      if (jy < 0 || jy >= nx) continue;
      const float* dr = dy + ((size_t)p * nx + jy) * COUT;
      for (int a = 0; a < COUT; ++a) acc += n.W2[(a * H + o) * KW + d] * dr[a];
    }
    const float hv = h1[t];
    dz1[t] = acc * (1.0f - hv * hv);
  }
}

// gradient of every parameter: one thread per parameter, fixed summation order
__global__ void k_grad(int H, const float* __restrict__ x, const float* __restrict__ h1,
                       const float* __restrict__ dz1, const float* __restrict__ dy, int P, int nx,
                       float* __restrict__ g) {
  const int n1 = H * CIN * KW, n2 = n1 + H, n3 = n2 + COUT * H * KW, np = n3 + COUT;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (i < n1) {
      const int o = i / (CIN * KW), c = (i / KW) % CIN, d = i % KW;
      for (int p = 0; p < P; ++p)
        for (int j = 0; j < nx; ++j) {
          const int jj = j + d - 2;
          if (jj < 0 || jj >= nx) continue;
          acc += (double)dz1[((size_t)p * nx + j) * H + o] * x[((size_t)p * nx + jj) * CIN + c];
        }
    } else if (i < n2) {
      const int o = i - n1;
      for (size_t q = 0; q < (size_t)P * nx; ++q) acc += dz1[q * H + o];
    } else if (i < n3) {
      const int r = i - n2, a = r / (H * KW), o = (r / KW) % H, d = r % KW;
      for (int p = 0; p < P; ++p)
        for (int j = 0; j < nx; ++j) {
          const int jj = j + d - 2;
          if (jj < 0 || jj >= nx) continue;
          acc += (double)dy[((size_t)p * nx + j) * COUT + a] * h1[((size_t)p * nx + jj) * H + o];
        }
    } else {
      const int a = i - n3;
      for (size_t q = 0; q < (size_t)P * nx; ++q) acc += dy[q * COUT + a];
    }
    g[i] = (float)acc;
  }
}

__global__ void k_sum(const float* __restrict__ a, size_t n, double scale, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
  double r = bsum(s, sh);
  if (threadIdx.x == 0) *out = r * scale;
}

// ------------------------------------------------ global linear form
// hidden = 0: one linear convolution over the whole slab,
//   y[p][j][a] = b[a] + sum_{c, d} W[a][c][d] x[p][j + d - (nx - 1)][c],
// d = 0 .. 2 nx - 2 (every cell sees every other cell), zero padding.
__global__ void k_lin_fwd(const float* __restrict__ th, int nx, const float* __restrict__ x, int P,
                          const float* __restrict__ t, float* __restrict__ y, float* __restrict__ dy,
                          float* __restrict__ se) {
  const int KWg = 2 * nx - 1;
  const float* W = th;
  const float* b = th + (size_t)COUT * CIN * KWg;
  const size_t total = (size_t)P * nx * COUT;
  const float inv = 1.0f / (float)total;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(q % COUT), j = (int)((q / COUT) % nx), p = (int)(q / ((size_t)COUT * nx));
    float acc = b[a];
    for (int jj = 0; jj < nx; ++jj) {
      const int d = jj - j + nx - 1;
      const float* xr = x + ((size_t)p * nx + jj) * CIN;
      for (int c = 0; c < CIN; ++c) acc += W[(a * CIN + c) * KWg + d] * xr[c];
    }
    if (y) y[q] = acc;
    if (t) {
      const float e = acc - t[q];
      dy[q] = 2.0f * e * inv;
      se[q] = e * e;
    }
  }
}

__global__ void k_lin_grad(int nx, const float* __restrict__ x, const float* __restrict__ dy, int P,
                           float* __restrict__ g) {
  const int KWg = 2 * nx - 1;
  const size_t nw = (size_t)COUT * CIN * KWg, np = nw + COUT;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < np; i += (size_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    if (i < nw) {
      const int a = (int)(i / (CIN * KWg)), c = (int)((i / KWg) % CIN), d = (int)(i % KWg);
      for (int p = 0; p < P; ++p)
        for (int j = 0; j < nx; ++j) {
          const int jj = j + d - (nx - 1);
          if (jj < 0 || jj >= nx) continue;
          acc += (double)dy[((size_t)p * nx + j) * COUT + a] * x[((size_t)p * nx + jj) * CIN + c];
        }
    } else {
      const int a = (int)(i - nw);
      for (size_t q = 0; q < (size_t)P * nx; ++q) acc += dy[q * COUT + a];
    }
    g[i] = (float)acc;
  }
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int np, float lr, float b1, float b2, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    m[i] = b1 * m[i] + (1 - b1) * gi;
    v[i] = b2 * v[i] + (1 - b2) * gi * gi;
    th[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + 1e-8f);
  }
}

// feature normalisation of stored pairs: x / sigma_p / cs_in, t / sigma_p / cs_out
__global__ void k_normalise(const float* __restrict__ xr, const float* __restrict__ tr, int P, int nx,
                            const float* __restrict__ sigma, const float* __restrict__ sc, float* __restrict__ xn,
                            float* __restrict__ tn) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < (size_t)P * nx; q += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(q / nx);
    const float s = sigma[p];
    for (int c = 0; c < CIN; ++c) xn[q * CIN + c] = xr[q * CIN + c] / s / sc[c];
    if (tr)
      for (int a = 0; a < COUT; ++a) tn[q * COUT + a] = tr[q * COUT + a] / s / sc[CIN + a];
  }
}

// z += sum_a c_{j,a} phi_a(v) M_j(v)
__global__ void k_lift(double* __restrict__ z, const float* __restrict__ c, const double* __restrict__ params, int N,
                       int nx, double h) {
  const size_t n3 = (size_t)N * N * N, len = n3 * nx;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / n3);
    double ph[NMOM];
    phis((int)(t % n3), N, h, ph);
    const double* pp = params + 5 * j;
    const double d1 = ph[1] - pp[1], d2 = ph[2] - pp[2], d3 = ph[3] - pp[3];
    const double M = pp[0] * pow(2.0 * 3.141592653589793 * pp[4], -1.5) * exp(-(d1 * d1 + d2 * d2 + d3 * d3) / (2.0 * pp[4]));
    const float* cj = c + j * COUT;
    z[t] += M * (cj[0] + cj[1] * ph[1] + cj[2] * ph[2] + cj[3] * ph[3] + cj[4] * ph[4]);
  }
}

int blocks_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 1216 ? (b > 0 ? b : 1) : 1216);
}

// loss and gradient on device arrays (used by training and by the ABI check)
lbo_status loss_grad_device(int H, const float* th, const float* x, const float* t, int P, int nx, float* h1,
                            float* dz1, float* y, float* dy, float* se, double* d_loss, float* g,
                            cudaStream_t s) {
  if (H == 0) {  // global linear convolution
    k_lin_fwd<<<blocks_for((size_t)P * nx * COUT), 256, 0, s>>>(th, nx, x, P, t, y, dy, se);
    k_lin_grad<<<blocks_for(param_count_nx(0, nx)), 256, 0, s>>>(nx, x, dy, P, g);
    k_sum<<<1, 1024, 0, s>>>(se, (size_t)P * nx * COUT, 1.0 / ((double)P * nx * COUT), d_loss);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LBO_OK : cuda_fail(e, "linear network loss/grad");
  }
  k_fwd1<<<blocks_for((size_t)P * nx * H), 256, 0, s>>>(th, H, x, P, nx, h1);
  k_fwd2<<<blocks_for((size_t)P * nx * COUT), 256, 0, s>>>(th, H, h1, P, nx, t, y, dy, se);
  k_bwd1<<<blocks_for((size_t)P * nx * H), 256, 0, s>>>(th, H, h1, dy, P, nx, dz1);
  k_grad<<<blocks_for((size_t)param_count(H)), 256, 0, s>>>(H, x, h1, dz1, dy, P, nx, g);
  k_sum<<<1, 1024, 0, s>>>(se, (size_t)P * nx * COUT, 1.0 / ((double)P * nx * COUT), d_loss);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "network loss/grad");
}

NetState* state(lbo_solver* S) { return (NetState*)S->netstate; }

}  // namespace

// z (already the sweep of v) += learned macroscopic correction
// sigma = RMS of the sweep moments (feature channels NMOM..NMOM+4) and the
// normalised features x / (sigma cs_in); one block
__global__ void k_feat_norm(float* __restrict__ feat, int nx, float* __restrict__ sc) {
  __shared__ double sh[32];
  double a = 0;
  for (int i = threadIdx.x; i < nx * 5; i += blockDim.x) {
    const double x = feat[(i / 5) * CIN + NMOM + i % 5];
    a += x * x;
  }
  const double tot = bsum(a, sh);
  __shared__ float sigma;
  if (threadIdx.x == 0) {
    sigma = (float)sqrt(tot / (5.0 * nx)) + 1e-30f;
    sc[CIN + COUT] = sigma;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nx * CIN; i += blockDim.x) feat[i] = feat[i] / sigma / sc[i % CIN];
}

// c = sigma cs_out (.) y
__global__ void k_corr_scale(float* __restrict__ corr, int nx, const float* __restrict__ sc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx * COUT; i += gridDim.x * blockDim.x)
    corr[i] *= sc[CIN + COUT] * sc[CIN + i % COUT];
}

// ns->r = v - A_T s (the operator without collisions)
static lbo_status transport_residual(lbo_solver* S, NetState* ns, const double* v, const double* s) {
  if (!ns->r) {
    cudaError_t e = cudaMalloc(&ns->r, sizeof(double) * S->len);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error_text("network: residual buffer");
      return LBO_ENOMEM;
    }
  }
  lbo_status st = solver_apply_op(S, s, ns->r, true, false);
  if (st != LBO_OK) return st;
  solver_axpby(S, ns->r, v, 1.0, -1.0);
  return LBO_OK;
}

static lbo_status upload_scales(NetState* ns) {
  if (!ns->dev_sc) {
    cudaError_t e = cudaMalloc(&ns->dev_sc, sizeof(float) * (CIN + COUT + 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error_text("network: scales");
      return LBO_ENOMEM;
    }
  }
  cudaError_t e = cudaMemcpy(ns->dev_sc, ns->scales, sizeof(float) * (CIN + COUT), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "network scales");
}

lbo_status network_correction(lbo_solver* S, const double* v, double* z) {
  NetState* ns = state(S);
  if (!ns || !ns->trained) return LBO_OK;
  cudaStream_t s = S->plan->stream;
  const int nx = S->nx, H = ns->hidden;
  lbo_status st = transport_residual(S, ns, v, z);
  if (st != LBO_OK) return st;
  k_cell_features<<<nx, 256, 0, s>>>(ns->r, z, nullptr, S->params, S->N, S->h, ns->feat, nullptr);
  k_feat_norm<<<1, 256, 0, s>>>(ns->feat, nx, ns->dev_sc);
  if (H == 0) {
    k_lin_fwd<<<blocks_for((size_t)nx * COUT), 256, 0, s>>>(ns->theta, nx, ns->feat, 1, nullptr, ns->corr, nullptr,
                                                          nullptr);
  } else {
    float* h1 = ns->corr + (size_t)nx * COUT;  // scratch after the outputs
    k_fwd1<<<blocks_for((size_t)nx * H), 256, 0, s>>>(ns->theta, H, ns->feat, 1, nx, h1);
    k_fwd2<<<blocks_for((size_t)nx * COUT), 256, 0, s>>>(ns->theta, H, h1, 1, nx, nullptr, ns->corr, nullptr, nullptr);
  }
  k_corr_scale<<<blocks_for((size_t)nx * COUT), 256, 0, s>>>(ns->corr, nx, ns->dev_sc);
  LBO_LAUNCH(S->plan, "net_lift", s, k_lift, blocks_for(S->len), 256, 0, z, ns->corr, S->params, S->N, nx, S->h);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "network correction");
}

bool network_collecting(const lbo_solver* S) {
  const NetState* ns = (const NetState*)S->netstate;
  return ns && ns->collecting && ns->pairs < ns->max_pairs;
}

// record a training pair (w = A z_k, z_k); s is scratch for sweep(w)
lbo_status network_record(lbo_solver* S, const double* w, const double* zk, double* s_scratch,
                          lbo_status (*sweep)(lbo_solver*, const double*, double*)) {
  NetState* ns = state(S);
  if (!ns || !ns->collecting || ns->pairs >= ns->max_pairs) return LBO_OK;
  lbo_status st = sweep(S, w, s_scratch);
  if (st == LBO_OK) st = transport_residual(S, ns, w, s_scratch);
  if (st != LBO_OK) return st;
  const int nx = S->nx;
  k_cell_features<<<nx, 256, 0, S->plan->stream>>>(ns->r, s_scratch, zk, S->params, S->N, S->h,
                                                    ns->store_x + (size_t)ns->pairs * nx * CIN,
                                                    ns->store_t + (size_t)ns->pairs * nx * COUT);
  ns->pairs++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "network record");
}

void free_network(lbo_solver* S) {
  NetState* ns = state(S);
  if (!ns) return;
  float* bufs[] = {ns->store_x, ns->store_t, ns->theta, ns->feat, ns->corr, ns->dev_sc};
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (ns->r) cudaFree(ns->r);
  delete ns;
  S->netstate = nullptr;
}

static NetState* ensure_state(lbo_solver* S, int hidden) {
  NetState* ns = state(S);
  if (!ns) {
    ns = new NetState();
    ns->hidden = -1;
    S->netstate = ns;
  }
  if (hidden >= 0 && ns->hidden != hidden) {
    if (ns->theta) cudaFree(ns->theta);
    ns->theta = nullptr;
    if (ns->corr) cudaFree(ns->corr);
    ns->corr = nullptr;
    ns->hidden = hidden;
  }
  return ns;
}

}  // namespace lbo

using namespace lbo;

extern "C" {

int lbo_network_param_count(int hidden) { return hidden > 0 ? param_count(hidden) : 0; }

lbo_status lbo_network_loss_grad(int hidden, const float* theta, const float* x, const float* t, int pairs, int nx,
                                 double* loss, float* grad) {
  if (hidden < 1 || !theta || !x || !t || pairs < 1 || nx < 1 || !grad) return LBO_EINVAL;
  const size_t a = (size_t)pairs * nx;
  float *h1 = nullptr, *dz1 = nullptr, *y = nullptr, *dy = nullptr, *se = nullptr;
  double* dl = nullptr;
  cudaError_t e = cudaMalloc(&h1, sizeof(float) * a * hidden);
  if (e == cudaSuccess) e = cudaMalloc(&dz1, sizeof(float) * a * hidden);
  if (e == cudaSuccess) e = cudaMalloc(&y, sizeof(float) * a * COUT);
  if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * a * COUT);
  if (e == cudaSuccess) e = cudaMalloc(&se, sizeof(float) * a * COUT);
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(double));
  lbo_status st = e == cudaSuccess ? loss_grad_device(hidden, theta, x, t, pairs, nx, h1, dz1, y, dy, se, dl, grad, 0)
                                   : cuda_fail(e, "network scratch");
  if (st == LBO_OK && loss) {
    e = cudaMemcpy(loss, dl, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_fail(e, "network loss copy");
  }
  void* bufs[] = {h1, dz1, y, dy, se, dl};
  for (void* p : bufs)
    if (p) cudaFree(p);
  return st;
}

lbo_status lbo_solver_collect(lbo_solver* S, int max_pairs) {
  if (!S || max_pairs < 0) return LBO_EINVAL;
  if (S->pb.kind != LBO_PROBLEM_SLAB) return LBO_EUNSUPPORTED;
  NetState* ns = ensure_state(S, 0);
  if (max_pairs == 0) {
    ns->collecting = false;
    return LBO_OK;
  }
  if (max_pairs != ns->max_pairs) {
    if (ns->store_x) cudaFree(ns->store_x);
    if (ns->store_t) cudaFree(ns->store_t);
    ns->store_x = ns->store_t = nullptr;
    cudaError_t e = cudaMalloc(&ns->store_x, sizeof(float) * (size_t)max_pairs * S->nx * CIN);
    if (e == cudaSuccess) e = cudaMalloc(&ns->store_t, sizeof(float) * (size_t)max_pairs * S->nx * COUT);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error_text("pair store allocation");
      return LBO_ENOMEM;
    }
    ns->max_pairs = max_pairs;
    ns->pairs = 0;
  }
  ns->collecting = true;
  return LBO_OK;
}

int lbo_solver_pair_count(lbo_solver* S) { return (S && S->netstate) ? state(S)->pairs : 0; }

lbo_status lbo_solver_train_network(lbo_solver* S, int hidden, int epochs, double lr, unsigned seed,
                                    double* final_loss) {
  if (!S || hidden < 0 || hidden > 256 || epochs < 1 || !(lr > 0)) return LBO_EINVAL;
  NetState* ns = ensure_state(S, hidden);
  const int P = ns->pairs, nx = S->nx;
  if (P < 1) {
    set_error_text("no training pairs collected");
    return LBO_EINVAL;
  }
  cudaStream_t s = S->plan->stream;
  const size_t a = (size_t)P * nx;
  // normalisation: per-pair sigma (RMS of the sweep moments) and channel scales
  std::vector<float> xr(a * CIN), tr(a * COUT), sig(P);
  cudaMemcpy(xr.data(), ns->store_x, sizeof(float) * xr.size(), cudaMemcpyDeviceToHost);
  cudaMemcpy(tr.data(), ns->store_t, sizeof(float) * tr.size(), cudaMemcpyDeviceToHost);
  std::vector<double> ch(CIN + COUT, 0.0);
  for (int p = 0; p < P; ++p) {
    double ss = 0;
    for (int j = 0; j < nx; ++j)
      for (int c = NMOM; c < NMOM + 5; ++c)
        ss += (double)xr[((size_t)p * nx + j) * CIN + c] * xr[((size_t)p * nx + j) * CIN + c];
    sig[p] = (float)std::sqrt(ss / (5.0 * nx)) + 1e-30f;
    for (int j = 0; j < nx; ++j) {
      for (int c = 0; c < CIN; ++c) {
        double v = xr[((size_t)p * nx + j) * CIN + c] / sig[p];
        ch[c] += v * v;
      }
      for (int c = 0; c < COUT; ++c) {
        double v = tr[((size_t)p * nx + j) * COUT + c] / sig[p];
        ch[CIN + c] += v * v;
      }
    }
  }
  for (int c = 0; c < CIN + COUT; ++c) ns->scales[c] = (float)std::sqrt(ch[c] / (double)a) + 1e-30f;
  const size_t np = param_count_nx(hidden, nx);
  std::vector<float> th0(np, 0.0f);
  unsigned st_rng = seed * 2654435761u + 12345u;
  auto urand = [&]() {
    st_rng = st_rng * 1664525u + 1013904223u;
    return ((st_rng >> 8) & 0xFFFFFF) / 16777216.0f - 0.5f;
  };
  const float s1 = 2.0f / std::sqrt((float)(CIN * KW)), s2 = 2.0f / std::sqrt((float)(hidden * KW));
  if (hidden > 0)
    for (size_t i = 0; i < np; ++i) th0[i] = urand() * ((int)i < hidden * CIN * KW + hidden ? s1 : s2);
  float *xn = nullptr, *tn = nullptr, *d_sig = nullptr, *d_sc = nullptr, *h1 = nullptr, *dz1 = nullptr, *y = nullptr,
        *dy = nullptr, *se = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  double* dl = nullptr;
  cudaError_t e = cudaSuccess;
  auto al = [&](float** p, size_t n) {
    if (e == cudaSuccess) e = cudaMalloc(p, sizeof(float) * n);
  };
  al(&xn, a * CIN);
  al(&tn, a * COUT);
  al(&d_sig, P);
  al(&d_sc, CIN + COUT);
  al(&h1, a * (hidden > 0 ? hidden : 1));
  al(&dz1, a * (hidden > 0 ? hidden : 1));
  al(&y, a * COUT);
  al(&dy, a * COUT);
  al(&se, a * COUT);
  al(&g, np);
  al(&m, np);
  al(&v, np);
  if (!ns->theta) al(&ns->theta, np);
  if (!ns->corr) al(&ns->corr, (size_t)nx * (COUT + (hidden > 0 ? hidden : 1)));
  if (!ns->feat) al(&ns->feat, (size_t)nx * CIN);
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(double));
  lbo_status result = LBO_OK;
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error_text("network training allocation");
    result = LBO_ENOMEM;
  } else {
    cudaMemcpy(d_sig, sig.data(), sizeof(float) * P, cudaMemcpyHostToDevice);
    cudaMemcpy(d_sc, ns->scales, sizeof(float) * (CIN + COUT), cudaMemcpyHostToDevice);
    cudaMemcpy(ns->theta, th0.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    cudaMemset(m, 0, sizeof(float) * np);
    cudaMemset(v, 0, sizeof(float) * np);
    k_normalise<<<blocks_for(a), 256, 0, s>>>(ns->store_x, ns->store_t, P, nx, d_sig, d_sc, xn, tn);
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f, c2 = 1.f;
    for (int ep = 0; ep < epochs && result == LBO_OK; ++ep) {
      result = loss_grad_device(hidden, ns->theta, xn, tn, P, nx, h1, dz1, y, dy, se, dl, g, s);
      c1 *= b1;
      c2 *= b2;
      k_adam<<<blocks_for(np), 256, 0, s>>>(ns->theta, g, m, v, (int)np, (float)lr, b1, b2, 1.f - c1, 1.f - c2);
    }
    if (result == LBO_OK) result = loss_grad_device(hidden, ns->theta, xn, tn, P, nx, h1, dz1, y, dy, se, dl, g, s);
    if (result == LBO_OK) result = upload_scales(ns);
    if (result == LBO_OK) ns->trained = true;
    if (result == LBO_OK && final_loss) {
      e = cudaMemcpyAsync(final_loss, dl, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) result = cuda_fail(e, "training");
    }
  }
  float* bufs[] = {xn, tn, d_sig, d_sc, h1, dz1, y, dy, se, g, m, v};
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (dl) cudaFree(dl);
  return result;
}

lbo_status lbo_solver_get_network(lbo_solver* S, int* hidden, float* params, float* scales) {
  if (!S || !hidden) return LBO_EINVAL;
  NetState* ns = state(S);
  if (!ns || !ns->trained) {
    *hidden = -1;
    return LBO_OK;
  }
  *hidden = ns->hidden;
  if (params) {
    cudaError_t e = cudaMemcpy(params, ns->theta, sizeof(float) * param_count_nx(ns->hidden, S->nx),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "get network");
  }
  if (scales) std::memcpy(scales, ns->scales, sizeof(ns->scales));
  return LBO_OK;
}

lbo_status lbo_solver_set_network(lbo_solver* S, int hidden, const float* params, const float* scales) {
  if (!S || hidden < 0 || hidden > 256 || !params || !scales) return LBO_EINVAL;
  if (S->pb.kind != LBO_PROBLEM_SLAB) return LBO_EUNSUPPORTED;
  NetState* ns = ensure_state(S, hidden);
  const size_t np = param_count_nx(hidden, S->nx);
  cudaError_t e = cudaSuccess;
  if (!ns->theta) e = cudaMalloc(&ns->theta, sizeof(float) * np);
  if (e == cudaSuccess && !ns->corr)
    e = cudaMalloc(&ns->corr, sizeof(float) * (size_t)S->nx * (COUT + (hidden > 0 ? hidden : 1)));
  if (e == cudaSuccess && !ns->feat) e = cudaMalloc(&ns->feat, sizeof(float) * (size_t)S->nx * CIN);
  if (e == cudaSuccess) e = cudaMemcpy(ns->theta, params, sizeof(float) * np, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "set network");
  std::memcpy(ns->scales, scales, sizeof(ns->scales));
  lbo_status st = upload_scales(ns);
  if (st != LBO_OK) return st;
  ns->trained = true;
  return LBO_OK;
}

int lbo_solver_network_param_count(lbo_solver* S, int hidden) {
  return S ? (int)param_count_nx(hidden, S->nx) : 0;
}

}  // extern "C"

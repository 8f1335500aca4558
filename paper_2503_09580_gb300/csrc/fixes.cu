// FP64 post-processing of an operator output: removal of the zero Fourier
// mode (the mass fix of Sec. 4.2, L^_0 = 0) and the projection onto zero
// mass, momentum and energy (least squares on the grid; the paper cites such
// a post-processing in Sec. 1 without fixing it).
#include <cmath>

#include "lbo_internal.h"

namespace lbo {

struct Gram5 {
  double ginv[25];
};

// One CTA per instance: FP64 block reduction of the five moments, then the
// correction, in place.
__global__ void __launch_bounds__(512) k_fixes(double* __restrict__ out, int N, double h, int mass_fix,
                                               int moment_fix, Gram5 G) {
  const int b = blockIdx.x;
  const size_t n3 = (size_t)N * N * N;
  double* x = out + (size_t)b * n3;
  __shared__ double red[5][16];
  double m[5] = {0, 0, 0, 0, 0};
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    int i3 = (int)(t % N), i2 = (int)((t / N) % N), i1 = (int)(t / ((size_t)N * N));
    double v1 = (i1 - N / 2) * h, v2 = (i2 - N / 2) * h, v3 = (i3 - N / 2) * h;
    double y = x[t];
    m[0] += y;
    m[1] += v1 * y;
    m[2] += v2 * y;
    m[3] += v3 * y;
    m[4] += (v1 * v1 + v2 * v2 + v3 * v3) * y;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 5; ++a) {
    double v = m[a];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[a][warp] = v;
  }
  __syncthreads();
  __shared__ double lam[5];
  if (threadIdx.x == 0) {
    double s[5];
    for (int a = 0; a < 5; ++a) {
      double v = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[a][w];
      s[a] = v;
    }
    if (moment_fix) {
      for (int a = 0; a < 5; ++a) {
        double v = 0;
        for (int c = 0; c < 5; ++c) v += G.ginv[a * 5 + c] * s[c];
        lam[a] = v;
      }
    } else {
      lam[0] = s[0] / (double)n3;
      for (int a = 1; a < 5; ++a) lam[a] = 0.0;
    }
  }
  __syncthreads();
  const double l0 = lam[0], l1 = lam[1], l2 = lam[2], l3 = lam[3], l4 = lam[4];
  for (size_t t = threadIdx.x; t < n3; t += blockDim.x) {
    int i3 = (int)(t % N), i2 = (int)((t / N) % N), i1 = (int)(t / ((size_t)N * N));
    double v1 = (i1 - N / 2) * h, v2 = (i2 - N / 2) * h, v3 = (i3 - N / 2) * h;
    x[t] -= l0 + l1 * v1 + l2 * v2 + l3 * v3 + l4 * (v1 * v1 + v2 * v2 + v3 * v3);
  }
}

// Gram matrix of {1, v1, v2, v3, |v|^2} on the grid, inverted on the host.
static void gram_inverse(int N, double h, double* ginv) {
  double Gm[5][10] = {};
  for (int i1 = 0; i1 < N; ++i1)
    for (int i2 = 0; i2 < N; ++i2)
      for (int i3 = 0; i3 < N; ++i3) {
        double v1 = (i1 - N / 2) * h, v2 = (i2 - N / 2) * h, v3 = (i3 - N / 2) * h;
        double f[5] = {1.0, v1, v2, v3, v1 * v1 + v2 * v2 + v3 * v3};
        for (int a = 0; a < 5; ++a)
          for (int c = 0; c < 5; ++c) Gm[a][c] += f[a] * f[c];
      }
  for (int a = 0; a < 5; ++a)
    for (int c = 0; c < 5; ++c) Gm[a][5 + c] = a == c ? 1.0 : 0.0;
  for (int col = 0; col < 5; ++col) {  // Gauss-Jordan with partial pivoting
    int piv = col;
    for (int r = col + 1; r < 5; ++r)
      if (std::fabs(Gm[r][col]) > std::fabs(Gm[piv][col])) piv = r;
    for (int c = 0; c < 10; ++c) std::swap(Gm[col][c], Gm[piv][c]);
    double d = Gm[col][col];
    for (int c = 0; c < 10; ++c) Gm[col][c] /= d;
    for (int r = 0; r < 5; ++r)
      if (r != col) {
        double f = Gm[r][col];
        for (int c = 0; c < 10; ++c) Gm[r][c] -= f * Gm[col][c];
      }
  }
  for (int a = 0; a < 5; ++a)
    for (int c = 0; c < 5; ++c) ginv[a * 5 + c] = Gm[a][5 + c];
}

lbo_status launch_fixes(lbo_plan* p, double* out, int B, int N, double h, cudaStream_t s, int* launches) {
  Gram5 G;
  gram_inverse(N, h, G.ginv);
  LBO_LAUNCH(p, "conservation_fix", s, k_fixes, B, 512, 0, out, N, h, p->mass_fix, p->moment_fix, G);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "conservation fix");
}

}  // namespace lbo

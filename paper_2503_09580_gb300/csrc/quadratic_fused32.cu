// Fused FP32 quadratic operator Q(f,f) (Eq. (2.14)) for N = 32.
//
// Kernels per application of a batch:
//   k_q32_head:  F = FFT(f) / N^3 (natural frequency order), one block per
//                instance;
//   k_q32_gain:  grid (G + 1) x batch.  Blocks x < G take a group of radial
//                nodes j; for each hemisphere node m they invert F E and
//                F conj(E) on chip (E the Nyquist-averaged phase multiplier
//                of alpha = pi g_j sigma_m / (2L)), park T+ in a per-block
//                scratch and accumulate 4 w_m T+ T- in real space (scratch);
//                after the m loop one forward transform and the
//                phi_j(|k|^2)-weighted accumulation into a per-group partial
//                spectrum.  Block x = G writes the loss term -f InvFFT(F omega).
//   k_q32_tail:  out += InvFFT(sum of the partial spectra).
// The scratch rows of a block are written and read by the thread that owns
// them (row pair (i1, q)), so they need no synchronisation; the working set
// of the resident blocks (2 x 128 KB each) stays in L2.
#include <cmath>

#include "fused32.cuh"
#include "lbo_internal.h"

namespace lbo {
namespace {
using namespace f32;

struct QArgs {
  const double* f;     // [B][N^3]
  cpx<float>* F;       // [B][F_H] FFT(f) / N^3
  const float* phi;    // [J][QMAX]: 4 pi^2 w_j B_j s_j / N^3
  const float* omega;  // [QMAX] / N^3
  const double* gsw;   // [J] radial nodes, then [M][3] sigma, then [M] w_m
  float* scratch;      // [(G+1) B][2][N^3]: T+ and the m-sum of w_m T+ T-
  cpx<float>* part;    // [G][B][F_H]
  double* out;         // [B][N^3]
  double L;
  int J, M, G, B, Q;
};

// F = FFT(f) / N^3
__global__ void __launch_bounds__(F_THREADS, 1) k_q32_head(QArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  const int b = blockIdx.x, t = threadIdx.x;
  const double* fb = a.f + (size_t)b * 32768;
  if (t < 512) {
    const int i1 = t >> 4, qq = t & 15;
    cpx<float> z[32];
#pragma unroll
    for (int i3 = 0; i3 < 32; ++i3)
      z[i3] = make_c((float)fb[(i1 * 32 + 2 * qq) * 32 + i3], (float)fb[(i1 * 32 + 2 * qq + 1) * 32 + i3]);
    fft32<false>(z);
    split_store(z, V + i1 * S_PLANE + qq * S_PAIR);
  }
  __syncthreads();
  axis_pass<2, false>(V);
  __syncthreads();
  const int i2 = t / F_HC, k3 = t % F_HC;
  cpx<float>* base = V + srow(i2) + k3;
  cpx<float> x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = base[i * S_PLANE];
  fft32<false>(x);
  cpx<float>* dst = a.F + (size_t)b * F_H + i2 * F_HC + k3;
  const float s = 1.0f / 32768.0f;
#pragma unroll
  for (int i = 0; i < 32; ++i) dst[i * F_ROW] = cscale(x[i], s);
}

// V = inverse axis 1 of F x E (CONJ: conj(E)); e[d*32 + k] the per-axis factors.
template <bool CONJ>
__device__ __forceinline__ void phase_axis1(cpx<float>* V, const cpx<float>* Fb, const cpx<float>* e) {
  const int t = threadIdx.x, i2 = t / F_HC, k3 = t % F_HC;
  const cpx<float> e23 = cmul(e[32 + i2], e[64 + k3]);
  const cpx<float>* src = Fb + i2 * F_HC + k3;
  cpx<float> x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const cpx<float> m = cmul(e[i], e23);
    x[i] = CONJ ? cmulc(src[i * F_ROW], m) : cmul(src[i * F_ROW], m);
  }
  fft32<true>(x);
  cpx<float>* base = V + srow(i2) + k3;
#pragma unroll
  for (int i = 0; i < 32; ++i) base[i * S_PLANE] = x[i];
}

// Scratch layout of a block: element (i3, r) of the row pair owned by thread
// t (< 512) at [(2 i3 + r) * 512 + t], so that a warp touches 128 contiguous
// bytes per access.
__device__ __forceinline__ void rows_store_tplus(const cpx<float>* V, float* Tp, int t) {
  const int i1 = t >> 4, qq = t & 15;
  cpx<float> z[32];
  load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
  fft32<true>(z);
#pragma unroll
  for (int i3 = 0; i3 < 32; ++i3) {
    Tp[(2 * i3) * 512 + t] = z[i3].x;
    Tp[(2 * i3 + 1) * 512 + t] = z[i3].y;
  }
}

__device__ __forceinline__ void rows_accumulate(const cpx<float>* V, const float* Tp, float* Pm, int t, float wq,
                                                bool first) {
  const int i1 = t >> 4, qq = t & 15;
  cpx<float> z[32];
  load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
  fft32<true>(z);
#pragma unroll
  for (int i3 = 0; i3 < 32; ++i3) {
    const int o0 = (2 * i3) * 512 + t, o1 = o0 + 512;
    const float v0 = wq * Tp[o0] * z[i3].x, v1 = wq * Tp[o1] * z[i3].y;
    Pm[o0] = first ? v0 : Pm[o0] + v0;
    Pm[o1] = first ? v1 : Pm[o1] + v1;
  }
}

__global__ void __launch_bounds__(F_THREADS, 1) k_q32_gain(QArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  __shared__ cpx<float> e[96];
  const int grp = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
  const cpx<float>* Fb = a.F + (size_t)b * F_H;
  const double* fb = a.f + (size_t)b * 32768;
  if (grp == a.G) {  // loss term: out = -f InvFFT(F omega)
    {
      const int i2 = t / F_HC, k3 = t % F_HC;
      const cpx<float>* src = Fb + i2 * F_HC + k3;
      cpx<float> x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = cscale(src[i * F_ROW], 32768.0f * __ldg(a.omega + ksq(i, i2, k3)));
      fft32<true>(x);
      cpx<float>* base = V + srow(i2) + k3;
#pragma unroll
      for (int i = 0; i < 32; ++i) base[i * S_PLANE] = x[i];
    }
    __syncthreads();
    axis_pass<2, true>(V);
    __syncthreads();
    if (t < 512) {
      const int i1 = t >> 4, qq = t & 15;
      cpx<float> z[32];
      load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
      fft32<true>(z);
      double* o0 = a.out + (size_t)b * 32768 + (i1 * 32 + 2 * qq) * 32;
      const double* f0 = fb + (i1 * 32 + 2 * qq) * 32;
#pragma unroll 4
      for (int i3 = 0; i3 < 32; ++i3) {
        o0[i3] = -f0[i3] * (double)z[i3].x;
        o0[32 + i3] = -f0[32 + i3] * (double)z[i3].y;
      }
    }
    return;
  }
  const int j0 = (a.J * grp) / a.G, j1 = (a.J * (grp + 1)) / a.G;
  float* Tp = a.scratch + ((size_t)grp * a.B + b) * 2 * 32768;
  float* Pm = Tp + 32768;
  const double* sig = a.gsw + a.J;
  const double* wm = sig + 3 * a.M;
  cpx<float>* acc = a.part + ((size_t)grp * a.B + b) * F_H;
  for (int j = j0; j < j1; ++j) {
    const double cj = 3.141592653589793 * a.gsw[j] / (2.0 * a.L);
    for (int m = 0; m < a.M; ++m) {
      __syncthreads();  // previous users of e[] and V are done
      if (t < 96) {     // per-axis factors exp(i alpha_d k), Nyquist: cos(16 alpha_d)
        const int d = t / 32, k = t % 32;
        // alpha_d k / pi, reduced to [-1, 1] in FP64, then sincospi in FP32
        double x = cj * sig[3 * m + d] * (double)(k == 16 ? 16 : (k < 16 ? k : k - 32)) / 3.141592653589793;
        x -= 2.0 * rint(0.5 * x);
        float s, c;
        sincospif((float)x, &s, &c);
        e[t] = k == 16 ? make_c(c, 0.0f) : make_c(c, s);
      }
      __syncthreads();
      const float wq = (float)(4.0 * wm[m]);
      // T+ : inverse of F E, parked in the scratch
      phase_axis1<false>(V, Fb, e);
      __syncthreads();
      axis_pass<2, true>(V);
      __syncthreads();
      if (t < 512) rows_store_tplus(V, Tp, t);
      __syncthreads();
      // T- : inverse of F conj(E); accumulate w_m T+ T-
      phase_axis1<true>(V, Fb, e);
      __syncthreads();
      axis_pass<2, true>(V);
      __syncthreads();
      if (t < 512) rows_accumulate(V, Tp, Pm, t, wq, m == 0);
    }
    // forward transform of the m-sum, phi_j-weighted accumulation
    __syncthreads();
    if (t < 512) {
      const int i1 = t >> 4, qq = t & 15;
      cpx<float> z[32];
#pragma unroll
      for (int i3 = 0; i3 < 32; ++i3) z[i3] = make_c(Pm[(2 * i3) * 512 + t], Pm[(2 * i3 + 1) * 512 + t]);
      fft32<false>(z);
      split_store(z, V + i1 * S_PLANE + qq * S_PAIR);
    }
    __syncthreads();
    axis_pass<2, false>(V);
    __syncthreads();
    {
      const int i2 = t / F_HC, k3 = t % F_HC;
      cpx<float>* base = V + srow(i2) + k3;
      cpx<float>* ac = acc + i2 * F_HC + k3;
      const float* ph = a.phi + (size_t)j * a.Q;
      cpx<float> x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = base[i * S_PLANE];
      fft32<false>(x);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const cpx<float> v = cscale(x[i], __ldg(ph + ksq(i, i2, k3)));
        ac[i * F_ROW] = j == j0 ? v : ac[i * F_ROW] + v;
      }
    }
  }
}

// out += InvFFT(sum of the partial gain spectra)
__global__ void __launch_bounds__(F_THREADS, 1) k_q32_tail(QArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  const int b = blockIdx.x, t = threadIdx.x;
  {
    const int i2 = t / F_HC, k3 = t % F_HC;
    cpx<float> x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = make_c(0.f, 0.f);
    for (int gi = 0; gi < a.G; ++gi) {
      const cpx<float>* src = a.part + ((size_t)gi * a.B + b) * F_H + i2 * F_HC + k3;
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = x[i] + src[i * F_ROW];
    }
    fft32<true>(x);
    cpx<float>* base = V + srow(i2) + k3;
#pragma unroll
    for (int i = 0; i < 32; ++i) base[i * S_PLANE] = x[i];
  }
  __syncthreads();
  axis_pass<2, true>(V);
  __syncthreads();
  if (t < 512) {
    const int i1 = t >> 4, qq = t & 15;
    cpx<float> z[32];
    load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
    fft32<true>(z);
    double* o0 = a.out + (size_t)b * 32768 + (i1 * 32 + 2 * qq) * 32;
#pragma unroll 4
    for (int i3 = 0; i3 < 32; ++i3) {
      o0[i3] += (double)z[i3].x;
      o0[32 + i3] += (double)z[i3].y;
    }
  }
}

}  // namespace

size_t quad_fused32_workspace_bytes(int B, int G) {
  return (size_t)B * F_H * 8 * (1 + (size_t)G) + (size_t)(G + 1) * B * 2 * 32768 * 4;
}

lbo_status run_quadratic_fused32(lbo_plan* p, const double* f, double* out, int B, void* ws, const double* d_gsw,
                                 int M, int G, int* launches) {
  cudaError_t e = upload_twiddles();
  if (e != cudaSuccess) return cuda_fail(e, "fused Q twiddles");
  const size_t sm = sizeof(cpx<float>) * S_TOTAL;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_q32_head, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_q32_gain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_q32_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  QArgs a{};
  a.f = f;
  a.F = (cpx<float>*)ws;
  a.part = a.F + (size_t)B * F_H;
  a.scratch = (float*)(a.part + (size_t)G * B * F_H);
  a.phi = p->d_phi32;
  a.omega = p->d_omega32;
  a.gsw = d_gsw;
  a.out = out;
  a.L = p->L;
  a.J = p->J;
  a.M = M;
  a.G = G;
  a.B = B;
  a.Q = 3 * 16 * 16 + 1;
  cudaStream_t s = p->stream;
  LBO_LAUNCH(p, "q32_head", s, k_q32_head, B, F_THREADS, sm, a);
  LBO_LAUNCH(p, "q32_gain", s, k_q32_gain, dim3(G + 1, B), F_THREADS, sm, a);
  LBO_LAUNCH(p, "q32_tail", s, k_q32_tail, B, F_THREADS, sm, a);
  *launches += 3;
  e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "fused Q launch");
}

}  // namespace lbo

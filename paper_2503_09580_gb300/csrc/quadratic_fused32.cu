// Fused FP32 quadratic operator Q(f,f) (Eq. (2.14)) for N = 32.
//
// Kernels per application of a batch:
//   k_q32_head:  F = FFT(f) / N^3 (natural frequency order), one block per
//                instance;
//   k_q32_gain:  grid (G + 1) x batch.  Blocks x < G take a group of radial
//                nodes j; for each hemisphere node m they invert F E and
//                F conj(E) on chip (E the Nyquist-averaged phase multiplier
//                of alpha = pi g_j sigma_m / (2L)), park T+ in tensor memory
//                and accumulate 4 w_m T+ T- in real space (tensor memory);
//                after the m loop one forward transform and the
//                phi_j(|k|^2)-weighted accumulation into a per-group partial
//                spectrum.  Block x = G writes the loss term -f InvFFT(F omega).
//   k_q32_tail:  out += InvFFT(sum of the partial spectra).
// T+ and the m-sum (128 KB each per block) are written and read only by the
// thread that owns their row pair (i1, q) (t < 512), so they live in that
// thread's TMEM lane: warp w (< 16) holds lanes 32 (w % 4) + lane, T+ in
// columns 128 (w / 4) + (0..63) and the m-sum in 128 (w / 4) + (64..127),
// column 2 i3 + r for element (i3, r) of the pair -- all 512 columns of the
// SM.  The dynamic shared memory keeps one gain block per SM, so the
// allocation never waits.
#include <cmath>

#include "fused32.cuh"
#include "lbo_internal.h"
#include "tmem.cuh"

namespace lbo {
namespace {
using namespace f32;

struct QArgs {
  const double* f;     // [B][N^3]
  cpx<float>* F;       // [B][F_H] FFT(f) / N^3
  const float* phi;    // [J][QMAX]: 4 pi^2 w_j B_j s_j / N^3
  const float* omega;  // [QMAX] / N^3
  const double* gsw;   // [J] radial nodes, then [M][3] sigma, then [M] w_m
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

static_assert(2 * sizeof(cpx<float>) * S_TOTAL > 228 * 1024, "gain blocks must not share an SM");
static_assert(128 * (512 / 32 / 4) == tmem::kColumns, "T+ and the m-sum fill TMEM exactly");

// T+ (TMEM columns tp .. tp + 63) <- inverse row transform of the row pair of thread t
__device__ __forceinline__ void rows_store_tplus(const cpx<float>* V, uint32_t tp, int t) {
  const int i1 = t >> 4, qq = t & 15;
  cpx<float> z[32];
  load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
  fft32<true>(z);
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // i3 = 4c .. 4c + 3
    uint32_t r[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      r[2 * e] = __float_as_uint(z[4 * c + e].x);
      r[2 * e + 1] = __float_as_uint(z[4 * c + e].y);
    }
    tmem::st8(tp + 8 * c, r);
  }
  tmem::wait_st();
}

// m-sum (columns pm .. pm + 63) (+)= w T+ T-, T- the inverse row transform
template <bool FIRST>
__device__ __forceinline__ void rows_accumulate(const cpx<float>* V, uint32_t tp, uint32_t pm, int t, float wq) {
  const int i1 = t >> 4, qq = t & 15;
  cpx<float> z[32];
  load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
  fft32<true>(z);
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // i3 = 4c .. 4c + 3
    uint32_t a[8];
    tmem::ld8(tp + 8 * c, a);
    tmem::wait_ld(a);
#pragma unroll
    for (int e = 0; e < 4; ++e) {  // a <- w T+ T-
      a[2 * e] = __float_as_uint(wq * __uint_as_float(a[2 * e]) * z[4 * c + e].x);
      a[2 * e + 1] = __float_as_uint(wq * __uint_as_float(a[2 * e + 1]) * z[4 * c + e].y);
    }
    if (!FIRST) {
      uint32_t s[8];
      tmem::ld8(pm + 8 * c, s);
      tmem::wait_ld(s);
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = __float_as_uint(__uint_as_float(s[k]) + __uint_as_float(a[k]));
    }
    tmem::st8(pm + 8 * c, a);
  }
  tmem::wait_st();
}

__global__ void __launch_bounds__(F_THREADS, 1) k_q32_gain(QArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  __shared__ cpx<float> e[96];
  __shared__ uint32_t tmem_slot;
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
  if (t < 32) tmem::alloc(&tmem_slot, tmem::kColumns);
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const uint32_t tbase = tmem_slot;
  const uint32_t tp = tmem::addr(tbase, 32u * ((t >> 5) & 3), 128u * (t >> 7)), pm = tp + 64;
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
      // T+ : inverse of F E, parked in tensor memory
      phase_axis1<false>(V, Fb, e);
      __syncthreads();
      axis_pass<2, true>(V);
      __syncthreads();
      if (t < 512) rows_store_tplus(V, tp, t);
      __syncthreads();
      // T- : inverse of F conj(E); accumulate w_m T+ T-
      phase_axis1<true>(V, Fb, e);
      __syncthreads();
      axis_pass<2, true>(V);
      __syncthreads();
      if (t < 512) {
        if (m == 0) rows_accumulate<true>(V, tp, pm, t, wq);
        else rows_accumulate<false>(V, tp, pm, t, wq);
      }
    }
    // forward transform of the m-sum, phi_j-weighted accumulation
    __syncthreads();
    if (t < 512) {
      const int i1 = t >> 4, qq = t & 15;
      cpx<float> z[32];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t s[8];
        tmem::ld8(pm + 8 * c, s);
        tmem::wait_ld(s);
#pragma unroll
        for (int e = 0; e < 4; ++e) z[4 * c + e] = make_c(__uint_as_float(s[2 * e]), __uint_as_float(s[2 * e + 1]));
      }
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
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (t < 32) tmem::dealloc(tbase, tmem::kColumns);
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

size_t quad_fused32_workspace_bytes(int B, int G) { return (size_t)B * F_H * 8 * (1 + (size_t)G); }

lbo_status run_quadratic_fused32(lbo_plan* p, const double* f, double* out, int B, void* ws, const double* d_gsw,
                                 int M, int G, int* launches) {
  cudaError_t e = upload_twiddles();
  if (e != cudaSuccess) return cuda_fail(e, "fused Q twiddles");
  const size_t sm = sizeof(cpx<float>) * S_TOTAL;
  raise_smem_limit((const void*)k_q32_head, sm);
  raise_smem_limit((const void*)k_q32_gain, sm);
  raise_smem_limit((const void*)k_q32_tail, sm);
  QArgs a{};
  a.f = f;
  a.F = (cpx<float>*)ws;
  a.part = a.F + (size_t)B * F_H;
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

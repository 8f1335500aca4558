// Helpers of the fused FP32 kernels for N = 32 (one block holds a whole
// instance's half spectrum, 32 x 32 x 17 complex, in shared memory; every
// axis pass is an in-register 32-point FFT per thread, 544 threads).
// Shared-memory index of (i1, i2, k3) = i1*561 + (i2/2)*35 + (i2%2)*17 + k3:
// the packed row pair (i1, q) occupies half rows 2q and 2q+1 (34 slots) of
// a 35-slot pair, planes are 561 slots apart.  With the odd pair stride the
// row pass (16 threads of one plane on 16 pairs) and with the odd plane
// stride the axis passes are free of shared-memory bank conflicts.
// Global spectra keep the natural index i1*544 + i2*17 + k3.
#pragma once
#include "lin_kernels.cuh"

namespace lbo {
namespace f32 {

constexpr int F_N = 32, F_HC = 17, F_ROW = 544, F_H = 32 * 544, F_THREADS = 544;
constexpr int S_PAIR = 35, S_PLANE = 16 * S_PAIR + 1, S_TOTAL = 32 * S_PLANE;

// offset of half row i2 inside a shared-memory plane
__device__ __forceinline__ int srow(int i2) { return (i2 >> 1) * S_PAIR + (i2 & 1) * F_HC; }

// x <- DFT_32(x) (forward: exp(-2 pi i nk/32); inverse: conjugate, unnormalised)
template <bool INV>
__device__ __forceinline__ void fft32(cpx<float> (&x)[32]) {
  cpx<float> y[32];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    cpx<float> v[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) v[n2] = x[n1 + 4 * n2];
    dft8<float, INV>(v);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
      if (n1 == 0 || k2 == 0) y[n1 * 8 + k2] = v[k2];
      else y[n1 * 8 + k2] = INV ? cmulc(v[k2], tw64<float>(2 * n1 * k2)) : cmul(v[k2], tw64<float>(2 * n1 * k2));
    }
  }
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    cpx<float> w[4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) w[n1] = y[n1 * 8 + k2];
    dft4<float, INV>(w);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) x[k2 + 8 * k1] = w[k1];
  }
}

// Forward row pass tail: z = FFT(x_a + i x_b) along i3 -> two half rows at dst[0..16], dst[17..33].
__device__ __forceinline__ void split_store(const cpx<float> (&z)[32], cpx<float>* dst) {
#pragma unroll
  for (int k = 0; k <= 16; ++k) {
    cpx<float> z1 = z[k], z2 = conjc(z[(32 - k) & 31]);
    cpx<float> d = z1 - z2;
    dst[k] = cscale(z1 + z2, 0.5f);
    dst[17 + k] = make_c(0.5f * d.y, -0.5f * d.x);
  }
}

// Inverse row pass head: two half rows -> packed z = X_a + i X_b on k = 0..31.
__device__ __forceinline__ void load_merge(const cpx<float>* src, cpx<float> (&z)[32]) {
#pragma unroll
  for (int k = 0; k <= 16; ++k) {
    cpx<float> a = src[k], b = src[17 + k];
    if (k == 0 || k == 16) {
      z[k] = make_c(a.x, b.x);
    } else {
      z[k] = make_c(a.x - b.y, a.y + b.x);
      z[32 - k] = make_c(a.x + b.y, b.x - a.y);  // conj(a) + i conj(b)
    }
  }
}

__device__ __forceinline__ int ksq(int k1, int k2, int k3) {
  int a = k1 < 16 ? k1 : k1 - 32, b = k2 < 16 ? k2 : k2 - 32;
  return a * a + b * b + k3 * k3;
}

// In-place axis pass over pencils of V: AXIS 2 -> pencil (i1, k3) along i2;
// AXIS 1 -> pencil (i2, k3) along i1.
template <int AXIS, bool INV>
__device__ __forceinline__ void axis_pass(cpx<float>* V) {
  const int t = threadIdx.x;
  const int a = t / F_HC, k3 = t % F_HC;
  cpx<float>* base = AXIS == 2 ? V + a * S_PLANE + k3 : V + srow(a) + k3;
  cpx<float> x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = base[AXIS == 2 ? srow(i) : i * S_PLANE];
  fft32<INV>(x);
#pragma unroll
  for (int i = 0; i < 32; ++i) base[AXIS == 2 ? srow(i) : i * S_PLANE] = x[i];
}


}  // namespace f32
}  // namespace lbo

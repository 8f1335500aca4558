// FP64 kernels of Q(f,f) (M-point form, Eq. (2.14)) for N = 32 with one
// thread per pencil and the transforms in registers, as the FP64 L kernels
// of lin_reg64.cuh; the spectra keep the layout of the generic kernels.
//
//   k_q_phase_table_r64   per-axis phase factors exp(i alpha_d k) of every
//                         radial and hemisphere node, once per application
//                         (they depend on no instance)
//   k_axis1_phase_r64     F E and F conj(E), inverse axis 1 of both
//   k_plane_inv_prod_r64  inverse axes 2 and 3 of both (T+ and T-) and the
//                         product 4 w_m T+ T-
#pragma once
#include "lin_reg64.cuh"

namespace lbo {
namespace r64 {

// tab[((j M + m) 3 + d) N + k] = exp(i alpha_d centred(k)), alpha_d = pi g_j
// sigma_(m,d) / (2 L); at the Nyquist index cos(alpha_d N / 2), the average
// of the two images.  gj: radial nodes [J], sig: hemisphere nodes [M][3].
// grid = J M, block = 3 N.
static __global__ void __launch_bounds__(3 * RN) k_q_phase_table_r64(const double* __restrict__ gj,
                                                                     const double* __restrict__ sig, int M,
                                                                     double pi, double two_l,
                                                                     cpx<double>* __restrict__ tab) {
  const int j = blockIdx.x / M, m = blockIdx.x % M, d = threadIdx.x / RN, k = threadIdx.x % RN;
  const double c = pi * gj[j] / two_l;
  const double al = c * sig[3 * m + d];
  cpx<double> v;
  if (k == RN / 2) {
    v = make_c(cos(al * (RN / 2)), 0.0);
  } else {
    double s, co;
    sincos(al * (double)centred<RN>(k), &s, &co);
    v = make_c(co, s);
  }
  tab[(size_t)blockIdx.x * 3 * RN + threadIdx.x] = v;
}

// For hemisphere node m = m0 + blockIdx.z of one radial node (tabj: its
// phase factors, [M][3][N]): W1 = InvFFT_1(F E / N^3), W2 = InvFFT_1(F
// conj(E) / N^3), E(k) = e1(k1) e2(k2) e3(k3), one column per thread; F E
// stays in registers while F conj(E) waits in shared memory.
// grid = (17, B, mb), block = 32.
static __global__ void __launch_bounds__(32) k_axis1_phase_r64(const cpx<double>* __restrict__ FH,
                                                               cpx<double>* __restrict__ W1b,
                                                               cpx<double>* __restrict__ W2b,
                                                               const cpx<double>* __restrict__ tabj, int m0,
                                                               size_t mstride) {
  __shared__ cpx<double> S[32][32];  // [k1][thread]
  const int b = blockIdx.y, t = threadIdx.x, col = blockIdx.x * 32 + t;
  const cpx<double>* mf = tabj + (size_t)(m0 + blockIdx.z) * 3 * RN;
  cpx<double>* W1 = W1b + blockIdx.z * mstride;
  cpx<double>* W2 = W2b + blockIdx.z * mstride;
  const size_t inst = (size_t)b * RN * RNC;
  const int p2 = col / RHC, k3 = col % RHC;
  const cpx<double> e23 = cscale(cmul(mf[RN + freq_of_pos<RN>(p2)], mf[2 * RN + k3]), 1.0 / (double)(RN * RN * RN));
  // F through shared memory, so that its loads are not all held in registers
  // next to the transform's (the warp fences bound the live ranges)
#pragma unroll
  for (int k = 0; k < 32; ++k) S[k][t] = FH[inst + (size_t)pos_of_freq<RN>(k) * RNC + col];
  __syncwarp();
  cpx<double> x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const cpx<double> f = S[k][t];
    const cpx<double> e = cmul(mf[k], e23);
    x[k] = cmul(f, e);
    S[k][t] = cmulc(f, e);
  }
  __syncwarp();
  reg::fft32<double, true>(x);
#pragma unroll
  for (int i = 0; i < 32; ++i) W1[inst + (size_t)i * RNC + col] = x[i];
#pragma unroll
  for (int k = 0; k < 32; ++k) x[k] = S[k][t];
  reg::fft32<double, true>(x);
#pragma unroll
  for (int i = 0; i < 32; ++i) W2[inst + (size_t)i * RNC + col] = x[i];
}

// Inverse axis 2 of one column of a plane buffer (rows [i2][pp][k3], row
// stride RSB) in place: a column k3 = 1..15, or (packed) the pair of
// columns 0 and 16 of a plane, whose result (x_0, x_16) of each row goes to
// the k3 = 0 slot (the layout of k_plane_mh_r64).
template <int RSB>
__device__ __forceinline__ void column_inverse(cpx<double>* col, bool packed) {
  cpx<double> x[32];
  if (packed) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const cpx<double> u = col[pos_of_freq<RN>(k) * RSB], v = col[pos_of_freq<RN>(k) * RSB + 16];
      x[k] = make_c(u.x - v.y, u.y + v.x);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) x[k] = col[pos_of_freq<RN>(k) * RSB];
  }
  reg::fft32<double, true>(x);
#pragma unroll
  for (int i = 0; i < 32; ++i) col[i * RSB] = x[i];
}

// Half rows ra, rb (after the inverse axis-2 pass) -> z = x_a + i x_b on i3.
__device__ __forceinline__ void rows_inverse(const cpx<double>* ra, const cpx<double>* rb, cpx<double> (&z)[32]) {
  {
    const cpx<double> a0 = ra[0], b0 = rb[0];  // (x_0, x_16) of each row
    z[0] = make_c(a0.x, b0.x);
    z[16] = make_c(a0.y, b0.y);
  }
#pragma unroll
  for (int k = 1; k < 16; ++k) {
    const cpx<double> u = ra[k], v = rb[k];
    z[k] = make_c(u.x - v.y, u.y + v.x);
    z[32 - k] = make_c(u.x + v.y, v.x - u.y);
  }
  reg::fft32<double, true>(z);
}

// For hemisphere node m0 + blockIdx.z (inputs and output offset by
// blockIdx.z): T+ and T- from the axis-1 results W1, W2 (inverse axes 2
// and 3), P = 4 w_m T+ T- (a real field [B][N][N][N]).  T+ of a row pair is
// parked in its own shared-memory slots while T- is formed; P is staged in
// the second buffer and stored coalesced.  grid = (N / PPC, B, mb), block =
// 16 PPC, shared memory 2 PlaneR<PPC>::BYTES.
template <int PPC>
__global__ void __launch_bounds__(PlaneR<PPC>::THREADS) k_plane_inv_prod_r64(const cpx<double>* __restrict__ W1b,
                                                                           const cpx<double>* __restrict__ W2b,
                                                                           double* __restrict__ Pb,
                                                                           const double* __restrict__ wm, int m0,
                                                                           size_t mstride, size_t pstride) {
  constexpr int RSB = PlaneR<PPC>::RSB, NREG = 15 * PPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* B1 = (cpx<double>*)smem_raw;
  cpx<double>* B2 = B1 + RN * RSB;
  const int b = blockIdx.y, i1_0 = blockIdx.x * PPC, t = threadIdx.x;
  const double scale = 4.0 * wm[m0 + blockIdx.z];  // phi_j carries 4 pi^2 w_j B_j s_j / N^3; Eq. (2.14): 16 pi^2
  const size_t plane0 = ((size_t)b * RN + i1_0) * RN * RHC;
  const cpx<double>* g1 = W1b + blockIdx.z * mstride + plane0;
  const cpx<double>* g2 = W2b + blockIdx.z * mstride + plane0;
  for (int e = t; e < PPC * RN * RHC; e += blockDim.x) {
    const int k3 = e % RHC, rest = e / RHC, p2 = rest % RN, pp = rest / RN;
    B1[p2 * RSB + pp * RHC + k3] = g1[e];
    B2[p2 * RSB + pp * RHC + k3] = g2[e];
  }
  __syncthreads();
  {
    const bool packed = t >= NREG;
    const int off = packed ? (t - NREG) * RHC : (t / 15) * RHC + 1 + t % 15;
    column_inverse<RSB>(B1 + off, packed);
    __syncwarp();  // one pencil's registers at a time
    column_inverse<RSB>(B2 + off, packed);
  }
  __syncthreads();
  {
    const int pp = t % PPC, qq = t / PPC;
    cpx<double>* ra1 = B1 + (2 * qq) * RSB + pp * RHC;
    cpx<double>* ra2 = B2 + (2 * qq) * RSB + pp * RHC;
    double* ta = (double*)ra1;  // T+ of row 2 qq (32 reals in the row's own 17 slots)
    double* tb = (double*)(ra1 + RSB);
    cpx<double> z[32];
    rows_inverse(ra1, ra1 + RSB, z);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      ta[i] = z[i].x;
      tb[i] = z[i].y;
    }
    __syncwarp();  // one row pair's registers at a time
    rows_inverse(ra2, ra2 + RSB, z);
    double* pa = (double*)ra2;
    double* pb = (double*)(ra2 + RSB);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      pa[i] = scale * ta[i] * z[i].x;
      pb[i] = scale * tb[i] * z[i].y;
    }
  }
  __syncthreads();
  double* P = Pb + blockIdx.z * pstride + ((size_t)b * RN + i1_0) * RN * RN;
  for (int e = t; e < PPC * RN * RN; e += blockDim.x) {
    const int i3 = e % RN, i2 = (e / RN) % RN, pp = e / (RN * RN);
    P[e] = ((const double*)(B2 + i2 * RSB + pp * RHC))[i3];
  }
}

}  // namespace r64
}  // namespace lbo

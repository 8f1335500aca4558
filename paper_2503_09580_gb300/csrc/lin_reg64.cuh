// FP64 kernels of the generic L[g] sequence for N = 32 with one thread per
// pencil: every 32-point transform runs in registers with compile-time
// twiddles (fft_reg.cuh, 388 FP64 instructions against 448 for the
// two-stage shared-memory transform of fft.cuh).  GB300's FP64 pipe issues
// about 1.7 lanes per clock per SM, so these kernels are bound by their
// FP64 instruction count alone; the other pipes are idle.  The spectra keep
// the layout of the generic kernels (axes 1 and 2 in the digit-reversed
// positions of fft.cuh, k3 natural), so the two sets mix freely.
//
//   k_uhat_octant_r64 u^_j of every instance on its (N/2+1)^3 octant: the
//                    weight and its DCT-I along all three axes in one block
//   k_mh_table_r64   M^h / 2 of every instance, once per application
//   k_plane_mh_r64   psi_j <- M^h psi_j between InvFFT and FFT of axes 2, 3
//                    (Algorithm 1, gain loop): the axis-2 columns, then per
//                    thread a pair of half rows merged into one complex row,
//                    inverse transform, x M^h, forward transform and split,
//                    all in registers, then the axis-2 columns forward
//   k_axis1_uhat_r64 psi_j = InvFFT_1(u^_j r^ / N^3), u^_j from its octant
//                    planes by a DCT-I along axis 1 (or from the cache)
//   k_axis1_acc_r64  L^+ (+)= phi_j FFT_1(psi^_j)
#pragma once
#include "fft_reg.cuh"
#include "lin_kernels.cuh"

namespace lbo {
namespace r64 {

constexpr int RN = 32, RHC = 17, RNC = RN * RHC;

// Shared memory of k_plane_mh_r64 for PPC planes: half rows [i2][pp][k3] with
// a padded row stride, which keeps the row pass (thread (pp, qq) = (t % PPC,
// t / PPC) on rows 2 qq, 2 qq + 1 of plane pp) free of bank conflicts: the
// eight threads of a 16-byte shared-memory phase land on distinct 16-byte
// bank groups when 2 RSB = 2 (mod 8) for PPC = 2 and 4 (mod 8) for PPC = 4
// (any RSB for PPC = 8).  16 PPC threads: every pass has exactly one pencil
// per thread (PPC even fills whole warps), since an idle lane costs as much
// FP64 issue as a busy one.
template <int PPC>
struct PlaneR {
  static_assert(PPC == 2 || PPC == 4 || PPC == 8, "planes per CTA");
  static constexpr int RSB = PPC * RHC + (PPC == 2 ? 3 : 2);
  static constexpr int THREADS = 16 * PPC;
  static constexpr size_t BYTES = sizeof(cpx<double>) * RN * RSB;
};

// mh[b][i1][i2][i3] = M^h(v) / 2 of instance b (the factor between the
// inverse and forward transforms of the gain loop, the same for every radial
// node; the 1/2 is the row split's, see below), formed as (e1 / 2 e2) e3
// from the separable factors of fill_mh_tables.  grid = B, block = 256.
static __global__ void __launch_bounds__(256) k_mh_table_r64(const double* __restrict__ params, double h,
                                                      double* __restrict__ mh) {
  __shared__ double eh[3 * RN];
  const int b = blockIdx.x;
  const InstanceParams q = load_params(params, b);
  fill_mh_tables<RN>(eh, q, h);
  double* dst = mh + (size_t)b * RN * RN * RN;
  for (int e = threadIdx.x; e < RN * RN * RN; e += blockDim.x) {
    const int i3 = e % RN, i2 = (e / RN) % RN, i1 = e / (RN * RN);
    dst[e] = ((0.5 * eh[i1]) * eh[RN + i2]) * eh[2 * RN + i3];
  }
}

// One pencil's DCT-I of length 17 in place: x_d at p[d * stride], d = 0..16,
// U(k) = sum_d c_d x_d cos(2 pi k d / 32) (c_0 = c_16 = 1, c_d = 2), by the
// pairing of DctPencil (d with 16 - d) and the same correctly rounded
// cosines as the plan's DCT table, in the same order; coefficients that are
// exactly 0 are skipped.
__device__ __forceinline__ void dct17_inplace(double* p, int stride) {
  double ev[8], od[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    const double x0 = p[d * stride], x1 = p[(16 - d) * stride];
    ev[d] = x0 + x1;
    od[d] = x0 - x1;
  }
  const double mid = p[8 * stride];
#pragma unroll
  for (int k = 0; k < RHC; ++k) {
    double acc = (k & 1) ? 0.0 : ((k & 2) ? -2.0 * mid : 2.0 * mid);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const double c = (d == 0 ? 1.0 : 2.0) * cos32((k * d) & 31);
      if (c != 0.0) acc += c * ((k & 1) ? od[d] : ev[d]);
    }
    p[k * stride] = acc;
  }
}

// u^_j = FFT(M^g phit_j) of one instance on its whole octant (Algorithm 1,
// precomputation of the gain kernel): the weight w(d) = rho (pi theta)^-3/2
// exp(-|d h|^2 / theta) phit_j(d), d in [0, 16]^3, formed as k_uhat_planes
// forms it, then the DCT-I along axes 3, 2 and 1 in shared memory.  Output
// up[b][k1][k2][k3], the octant layout of the Maxwellian cache.
// grid = B, block = 320 (289 pencils per pass).
static __global__ void __launch_bounds__(320) k_uhat_octant_r64(const double* __restrict__ params,
                                                                const double* __restrict__ phit, double h,
                                                                double* __restrict__ up) {
  constexpr int HC2 = RHC * RHC, HC3 = HC2 * RHC;
  __shared__ double W[HC3];
  __shared__ double mg[RHC + 1];  // mg[17] = rho (pi theta)^-3/2
  const int b = blockIdx.x, t = threadIdx.x;
  const double rho = params[5 * b], theta = params[5 * b + 4];
  if (t < RHC) {
    const double x = t * h;
    mg[t] = exp(-(x * x) / theta);
  } else if (t == RHC) {
    mg[RHC] = rho * pow(3.141592653589793 * theta, -1.5);
  }
  __syncthreads();
  for (int e = t; e < HC3; e += blockDim.x) {
    const int d3 = e % RHC, d2 = (e / RHC) % RHC, d1 = e / HC2;
    const double w = mg[RHC] * (mg[d1] * mg[d2]) * mg[d3];
    W[e] = w * phit[((size_t)d1 * RN + d2) * RN + d3];
  }
  __syncthreads();
  if (t < HC2) dct17_inplace(W + t * RHC, 1);  // axis 3: pencil (d1, d2)
  __syncthreads();
  if (t < HC2) dct17_inplace(W + (t / RHC) * HC2 + t % RHC, RHC);  // axis 2: pencil (d1, k3)
  __syncthreads();
  if (t < HC2) dct17_inplace(W + t, HC2);  // axis 1: pencil (k2, k3)
  __syncthreads();
  double* dst = up + (size_t)b * HC3;
  for (int e = t; e < HC3; e += blockDim.x) dst[e] = W[e];
}

// grid = (N / PPC, B), block = PlaneR<PPC>::THREADS; src [B][N][N][N/2+1]
// (axis 1 spatial, axis 2 in positions) is transformed in place.
//
// Axis-2 pencils: columns k3 = 1..15 of every plane one per thread; the
// columns k3 = 0 and 16, which hold the transforms of real sequences
// (Hermitian along k2), share one complex transform per plane,
// Z = X_0 + i X_16.  Between the two axis-2 passes that pair lives in the
// k3 = 0 slot as (x_0, x_16) of each row; the row pass reads and writes it
// there, after the forward row transform at half scale so that the
// forward column split needs no multiplication:
//   X_0(k) = Z(k) + conj Z(-k),  X_16(k) = -i (Z(k) - conj Z(-k)).
template <int PPC>
__global__ void __launch_bounds__(PlaneR<PPC>::THREADS) k_plane_mh_r64(const double* __restrict__ mh,
                                                                     cpx<double>* __restrict__ src) {
  constexpr int RSB = PlaneR<PPC>::RSB, NREG = 15 * PPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* Bs = (cpx<double>*)smem_raw;
  const int b = blockIdx.y, i1_0 = blockIdx.x * PPC, t = threadIdx.x;
  cpx<double>* gsrc = src + ((size_t)b * RN + i1_0) * RN * RHC;
  for (int e = t; e < PPC * RN * RHC; e += blockDim.x) {
    const int k3 = e % RHC, rest = e / RHC, p2 = rest % RN, pp = rest / RN;
    Bs[p2 * RSB + pp * RHC + k3] = gsrc[e];
  }
  __syncthreads();
  // axis-2 pencil of this thread: column k3 = 1 + t % 15 of plane t / 15, or
  // (the last PPC threads) the packed pair of columns 0 and 16 of plane t - NREG
  const bool packed = t >= NREG;
  cpx<double>* col = packed ? Bs + (t - NREG) * RHC : Bs + (t / 15) * RHC + 1 + t % 15;
  {  // inverse axis 2
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
  __syncthreads();
  {  // rows 2 qq (real part) and 2 qq + 1 (imaginary part) of plane pp
    const int pp = t % PPC, qq = t / PPC;
    cpx<double>* ra = Bs + (2 * qq) * RSB + pp * RHC;
    cpx<double>* rb = ra + RSB;
    cpx<double> z[32];
    {
      const cpx<double> a0 = ra[0], b0 = rb[0];  // (x_0, x_16) of each row
      z[0] = make_c(a0.x, b0.x);
      z[16] = make_c(a0.y, b0.y);
    }
#pragma unroll
    for (int k = 1; k < 16; ++k) {
      const cpx<double> u = ra[k], v = rb[k];
      z[k] = make_c(u.x - v.y, u.y + v.x);       // X_a + i X_b
      z[32 - k] = make_c(u.x + v.y, v.x - u.y);  // conj(X_a) + i conj(X_b)
    }
    reg::fft32<double, true>(z);
    // x M^h / 2 (the 1/2 of the split below)
    const double* ma = mh + (((size_t)b * RN + i1_0 + pp) * RN + 2 * qq) * RN;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      z[i].x *= __ldg(ma + i);
      z[i].y *= __ldg(ma + RN + i);
    }
    reg::fft32<double, false>(z);
    // k3 = 0 and 16 at half scale: X_a(0) / 2 = Re z(0), and so on
    ra[0] = make_c(z[0].x, z[16].x);
    rb[0] = make_c(z[0].y, z[16].y);
#pragma unroll
    for (int k = 1; k < 16; ++k) {
      const cpx<double> z1 = z[k], z2 = z[32 - k];
      ra[k] = make_c(z1.x + z2.x, z1.y - z2.y);  // z1 + conj(z2)
      rb[k] = make_c(z1.y + z2.y, z2.x - z1.x);  // (z1 - conj(z2)) / i
    }
  }
  __syncthreads();
  {  // forward axis 2
    cpx<double> x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = col[i * RSB];
    reg::fft32<double, false>(x);
    if (packed) {
#pragma unroll
      for (int k = 0; k <= 16; ++k) {
        const int m = (32 - k) & 31;
        const cpx<double> zk = x[k], zm = x[m];
        const double sx = zk.x + zm.x, dy = zk.y - zm.y, sy = zk.y + zm.y, dx = zm.x - zk.x;
        col[pos_of_freq<RN>(k) * RSB] = make_c(sx, dy);
        col[pos_of_freq<RN>(k) * RSB + 16] = make_c(sy, dx);
        if (k != 0 && k != 16) {
          col[pos_of_freq<RN>(m) * RSB] = make_c(sx, -dy);
          col[pos_of_freq<RN>(m) * RSB + 16] = make_c(sy, -dx);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < 32; ++k) col[pos_of_freq<RN>(k) * RSB] = x[k];
    }
  }
  __syncthreads();
  for (int e = t; e < PPC * RN * RHC; e += blockDim.x) {
    const int k3 = e % RHC, rest = e / RHC, p2 = rest % RN, pp = rest / RN;
    gsrc[e] = Bs[p2 * RSB + pp * RHC + k3];
  }
}

// Column (p2, k3) of the half spectrum: |k2| of position p2.
__device__ __forceinline__ int abs_k2(int p2) {
  const int k2 = centred<RN>(freq_of_pos<RN>(p2));
  return k2 < 0 ? -k2 : k2;
}

// psi_j = InvFFT_1(u^_j r^ * scale), one column per thread.  CACHED: u^_j
// read whole from its cached octant up[b][|k1|][|k2|][k3]; otherwise its
// axis-1 DCT-I is formed here from the octant planes up[b][d1][|k2|][k3]
// (axes 3 and 2 done by k_uhat_planes), with the pairing of DctPencil.
// grid = (17, B), block = 32: columns col = 32 blockIdx.x + threadIdx.x.
template <bool CACHED>
__global__ void __launch_bounds__(32) k_axis1_uhat_r64(Axis1Args a, const cpx<double>* __restrict__ src,
                                                        cpx<double>* __restrict__ dst) {
  const int b = blockIdx.y, col = blockIdx.x * 32 + threadIdx.x;
  const size_t inst = (size_t)b * RN * RNC;
  const int p2 = col / RHC, k3 = col % RHC, k2 = abs_k2(p2);
  constexpr size_t HC2 = (size_t)RHC * RHC;
  const double* up = (const double*)a.uplanes + (size_t)b * HC2 * RHC + (size_t)k2 * RHC + k3;
  const double sc = a.scale;
  double U[RHC];
  if constexpr (CACHED) {
#pragma unroll
    for (int k = 0; k < RHC; ++k) U[k] = up[k * HC2] * sc;
  } else {
    double ev[8], od[8];
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const double x0 = up[d * HC2], x1 = up[(16 - d) * HC2];
      ev[d] = x0 + x1;
      od[d] = x0 - x1;
    }
    const double mid = up[8 * HC2];
    // coefficients c_d cos(2 pi k d / 32) as the plan's DCT table holds them
    // (the same correctly rounded cosines); the zero ones are skipped
#pragma unroll
    for (int k = 0; k < RHC; ++k) {
      double acc = (k & 1) ? 0.0 : ((k & 2) ? -2.0 * mid : 2.0 * mid);
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        const double c = (d == 0 ? 1.0 : 2.0) * cos32((k * d) & 31);
        if (c != 0.0) acc += c * ((k & 1) ? od[d] : ev[d]);
      }
      U[k] = acc * sc;
    }
  }
  cpx<double> x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) x[k] = cscale(src[inst + (size_t)pos_of_freq<RN>(k) * RNC + col], U[k <= 16 ? k : 32 - k]);
  reg::fft32<double, true>(x);
#pragma unroll
  for (int i = 0; i < 32; ++i) dst[inst + (size_t)i * RNC + col] = x[i];
}

// L^+ (+)= table(|k|^2) FFT_1(psi^_j), one column per thread (first: store).
// grid = (17, B), block = 32.
static __global__ void __launch_bounds__(32) k_axis1_acc_r64(Axis1Args a, const cpx<double>* __restrict__ src,
                                                       cpx<double>* __restrict__ dst) {
  const int b = blockIdx.y, col = blockIdx.x * 32 + threadIdx.x;
  const size_t inst = (size_t)b * RN * RNC;
  const int p2 = col / RHC, k3 = col % RHC, k2 = centred<RN>(freq_of_pos<RN>(p2));
  const int q23 = k2 * k2 + k3 * k3;
  const double* tab = (const double*)a.table;
  cpx<double> x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = src[inst + (size_t)i * RNC + col];
  reg::fft32<double, false>(x);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int c = k < 16 ? k : k - 32;
    const cpx<double> v = cscale(x[k], tab[c * c + q23]);
    cpx<double>* o = dst + inst + (size_t)pos_of_freq<RN>(k) * RNC + col;
    *o = a.first ? v : *o + v;
  }
}

}  // namespace r64
}  // namespace lbo

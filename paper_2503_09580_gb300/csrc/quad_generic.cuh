// The generic launch sequence of Q(f,f) (M-point form, Eq. (2.14)),
// shared by the translation units that instantiate it for their transform
// precisions (quadratic.cu: FP64 and FP32; quad_x2.cu: the two-fold forms).
//
// With F = FFT(f), for every radial node g_j and hemisphere node sigma_m,
// alpha = pi g_j sigma_m / (2L) and the phase multiplier
// E(k) = prod_d e^{i alpha_d k_d} (cos(alpha_d N/2) at the Nyquist index,
// the average over the two images):
//   T+ = InvFFT(F E),  T- = InvFFT(F conj(E))     (both real fields)
//   T+ T- = A_c^2 - B_s^2, the real-space form of I_{j,k,m}
//   Q^+ = 16 pi^2 sum_j w_j B(g_j) s_{j,k} FFT( sum_m w_m T+ T- )
//   Q   = InvFFT(Q^+) - f InvFFT(F omega).
// The sum over m is taken in real space before the forward transform of
// each j (the transform is linear), so one application costs 2 J M inverse
// transforms + J forward transforms + 4.
#pragma once
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "lbo_internal.h"
#include "lin_kernels.cuh"
#include "quad_reg64.cuh"

namespace lbo {

struct QuadState {
  int p = 0;                   // hemisphere order of the cached rule
  std::vector<double> sig, wm;  // M x 3, M
  // loss multiplier of Eq. (2.16) per half-spectrum position, in the
  // transform precision of omq_prec, for hemisphere order omq_p
  void* d_omq = nullptr;
  int omq_prec = -1, omq_p = -1;
  const void* omq_tables = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* d_gsw = nullptr;      // device copy: radial nodes, sigma, w_m (fused path)
  int gsw_p = -1;
  const void* gsw_plan_tables = nullptr;
};

template <int N>
struct PPCq { static constexpr int v = N == 16 ? 8 : (N == 32 ? 4 : (N == 24 ? 4 : (N == 48 ? 2 : 1))); };

// F (after all three forward passes) -> x E and x conj(E), inverse axis 1 of
// both, for hemisphere node m0 + blockIdx.z: alpha_d = c sigma_(m,d), results
// at W1, W2 + blockIdx.z * mstride.
template <typename T, int N, int CW>
__global__ void __launch_bounds__(256) k_axis1_phase(const cpx<T>* __restrict__ FH, cpx<T>* __restrict__ W1b,
                                                     cpx<T>* __restrict__ W2b, const double* __restrict__ sig,
                                                     int m0, double cj, size_t mstride) {
  constexpr int HC = N / 2 + 1, NC = N * HC;
  __shared__ __align__(16) cpx<T> S1[N * CW];
  __shared__ __align__(16) cpx<T> S2[N * CW];
  __shared__ cpx<double> mf[3 * N];  // per-axis factors, indexed by cyclic frequency
  __shared__ cpx<T> mfT[is_twofold<T>::value ? 3 * N : 1];  // the same in T (two-fold forms)
  const int b = blockIdx.y, c0 = blockIdx.x * CW, m = m0 + blockIdx.z;
  const double al1 = cj * sig[3 * m], al2 = cj * sig[3 * m + 1], al3 = cj * sig[3 * m + 2];
  cpx<T>* W1 = W1b + blockIdx.z * mstride;
  cpx<T>* W2 = W2b + blockIdx.z * mstride;
  const size_t inst = (size_t)b * N * NC;
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
    const int d = t / N, k = t % N;
    const double al = d == 0 ? al1 : (d == 1 ? al2 : al3);
    if (k == N / 2) {
      mf[t] = make_c(cos(al * (N / 2)), 0.0);
    } else {
      double s, c;
      sincos(al * (double)centred<N>(k), &s, &c);
      mf[t] = make_c(c, s);
    }
    if constexpr (is_twofold<T>::value) mfT[t] = make_c(T(mf[t].x), T(mf[t].y));
  }
  __syncthreads();
  const T inv_n3 = T(1.0 / ((double)N * N * N));
  for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
    const int c = t % CW, r = t / CW, col = c0 + c;
    if constexpr (is_twofold<T>::value) {
      // the phase product and both multiplications in T (no FP64 per point)
      if (col < NC) {
        const int p2 = col / HC, k3 = col % HC;
        const cpx<T> e = cscale(cmul(cmul(mfT[freq_of_pos<N>(r)], mfT[N + freq_of_pos<N>(p2)]), mfT[2 * N + k3]),
                                inv_n3);
        const cpx<T> f = FH[inst + (size_t)r * NC + col];
        S1[t] = cmul(f, e);
        S2[t] = cmulc(f, e);
      } else {
        S1[t] = make_c((T)0, (T)0);
        S2[t] = make_c((T)0, (T)0);
      }
      continue;
    }
    if (col < NC) {
      const int p2 = col / HC, k3 = col % HC;
      // 1/N^3 normalises the (unnormalised) inverse transforms of T+ and T-
      const cpx<double> e = cscale(cmul(cmul(mf[freq_of_pos<N>(r)], mf[N + freq_of_pos<N>(p2)]), mf[2 * N + k3]),
                                   1.0 / ((double)N * N * N));
      const cpx<T> f = FH[inst + (size_t)r * NC + col];
      const cpx<double> fd = make_c((double)f.x, (double)f.y);
      const cpx<double> a = cmul(fd, e), bb = cmulc(fd, e);
      S1[t] = make_c((T)a.x, (T)a.y);
      S2[t] = make_c((T)bb.x, (T)bb.y);
    } else {
      S1[t] = make_c((T)0, (T)0);
      S2[t] = make_c((T)0, (T)0);
    }
  }
  __syncthreads();
  smem_fft<T, N, true, true>(S1, CW, 1, CW);
  smem_fft<T, N, true, true>(S2, CW, 1, CW);
  for (int t = threadIdx.x; t < N * CW; t += blockDim.x) {
    const int c = t % CW, r = t / CW;
    if (c0 + c >= NC) continue;
    const size_t o = inst + (size_t)r * NC + c0 + c;
    W1[o] = S1[t];
    W2[o] = S2[t];
  }
}

// Inverse planes of W1, W2 -> T+, T-; P = 4 w_m T+ T- (real field, T) for
// hemisphere node m0 + blockIdx.z (inputs and output offset by blockIdx.z).
template <typename T, int N, int PPC>
__global__ void __launch_bounds__(256) k_plane_inv_prod(const cpx<T>* __restrict__ W1b, const cpx<T>* __restrict__ W2b,
                                                        T* __restrict__ Pb, const double* __restrict__ wm, int m0,
                                                        size_t mstride, size_t pstride) {
  const cpx<T>* W1 = W1b + blockIdx.z * mstride;
  const cpx<T>* W2 = W2b + blockIdx.z * mstride;
  T* P = Pb + blockIdx.z * pstride;
  // 4 w_m: phi_j carries 4 pi^2 w_j B_j s_j / N^3, Eq. (2.14) needs 16 pi^2
  const double scale = 4.0 * wm[m0 + blockIdx.z];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int E = PlaneSmem<T, N, PPC>::A_ELEMS + PlaneSmem<T, N, PPC>::B_ELEMS;
  cpx<T>* A1 = (cpx<T>*)smem_raw;
  cpx<T>* B1 = A1 + PlaneSmem<T, N, PPC>::A_ELEMS;
  cpx<T>* A2 = A1 + E;
  cpx<T>* B2 = A2 + PlaneSmem<T, N, PPC>::A_ELEMS;
  const int b = blockIdx.y, i1_0 = blockIdx.x * PPC;
  plane_load_B<T, N, PPC>(B1, W1, b, i1_0);
  plane_inverse_to_A<T, N, PPC>(A1, B1);
  plane_load_B<T, N, PPC>(B2, W2, b, i1_0);
  plane_inverse_to_A<T, N, PPC>(A2, B2);
  const T sc = (T)scale;
  for (int t = threadIdx.x; t < PPC * (N / 2) * N; t += blockDim.x) {
    const int i3 = t % N, rest = t / N, qq = rest % (N / 2), pp = rest / (N / 2);
    const cpx<T> zp = A1[(pp * (N / 2) + qq) * N + i3], zm = A2[(pp * (N / 2) + qq) * N + i3];
    const size_t o = (((size_t)b * N + i1_0 + pp) * N + 2 * qq) * N + i3;
    P[o] = sc * zp.x * zm.x;
    P[o + N] = sc * zp.y * zm.y;
  }
}

// Ps (+)= sum over the chunk's hemisphere nodes of P_m, in the order of m
template <typename T>
__global__ void k_sum_m(const T* __restrict__ Pm, T* __restrict__ Ps, int mb, size_t pstride, size_t total,
                        int first) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    T acc = first ? Pm[t] : Ps[t] + Pm[t];
    for (int z = 1; z < mb; ++z) acc += Pm[z * pstride + t];
    Ps[t] = acc;
  }
}

// hemisphere nodes per launch: all M, unless their buffers would pass 1 GiB
inline int q_chunk(int B, int M, int N, size_t rb) {
  const size_t H = (size_t)N * N * (N / 2 + 1), n3 = (size_t)N * N * N;
  const size_t per_m = (size_t)B * (2 * H * 2 * rb + n3 * rb);
  const size_t cap = (size_t)1 << 30;
  int mb = (int)std::max<size_t>(1, cap / std::max<size_t>(per_m, 1));
  return std::min(mb, std::max(M, 1));
}

// out = Q+ - f u  (FP64)
template <typename T, int N>
__global__ void k_combine_q(const double* __restrict__ f, const T* __restrict__ Qp, const T* __restrict__ uu,
                            double* __restrict__ out, size_t total) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
    out[t] = (double)Qp[t] - f[t] * (double)uu[t];
}

template <typename K>
inline void smem_attr(K kernel, size_t bytes) {
  raise_smem_limit((const void*)kernel, bytes);
}

template <typename T, int N>
static lbo_status run_quadratic(lbo_plan* p, QuadState* qs, const double* f, double* out, int B, const T* phi,
                         const T* omg, const T* omg3 = nullptr) {
  // 32-byte complex numbers (pairs of FP64): half the planes per block and
  // half the axis-1 tile, so that k_plane_inv_prod's two plane buffers and
  // k_axis1_phase's two tiles stay within the shared memory of a block
  constexpr bool wide = sizeof(cpx<T>) > 16;
  constexpr int PPC = wide && PPCq<N>::v > 1 ? PPCq<N>::v / 2 : PPCq<N>::v, CW = wide ? 16 : 32, HC = N / 2 + 1;
  const size_t H = (size_t)N * N * HC, n3 = (size_t)N * N * N;
  const int Q = 3 * (N / 2) * (N / 2) + 1;
  cudaStream_t s = p->stream;
  cpx<T>* FH = (cpx<T>*)qs->ws;
  cpx<T>* W1 = FH + (size_t)B * H;
  cpx<T>* W2 = W1 + (size_t)B * H;
  cpx<T>* QH = W2 + (size_t)B * H;
  T* Ps = (T*)(QH + (size_t)B * H);
  T* R1 = Ps + (size_t)B * n3;
  T* R2 = R1 + (size_t)B * n3;
  static_assert(2 * PlaneSmem<T, N, PPC>::BYTES <= 227 * 1024, "k_plane_inv_prod: shared memory of a block");
  static_assert(2 * N * CW * sizeof(cpx<T>) + 3 * N * (sizeof(cpx<double>) + sizeof(cpx<T>)) <= 227 * 1024,
                "k_axis1_phase: shared memory of a block");
  const size_t sm = PlaneSmem<T, N, PPC>::BYTES;
  const dim3 gp(N / PPC, B), ga((N * HC + CW - 1) / CW, B), blk(256);
  auto kf_real = k_plane_fwd<T, N, PPC, SRC_REAL64>;
  auto kf_t = k_plane_fwd<T, N, PPC, SRC_REALT>;
  auto ki_real = k_plane_inv<T, N, PPC, INV_TO_REAL>;
  auto ka_fwd = k_axis1<T, N, CW, AX_FWD_STORE>;
  auto ka_mult = k_axis1<T, N, CW, AX_FWD_MULT_INV>;
  auto ka_mult3 = k_axis1<T, N, CW, AX_FWD_MULT3_INV>;
  auto ka_acc = k_axis1<T, N, CW, AX_FWD_ACC>;
  auto ka_inv = k_axis1<T, N, CW, AX_INV_STORE>;
  auto ka_ph = k_axis1_phase<T, N, CW>;
  auto kp_prod = k_plane_inv_prod<T, N, PPC>;
  auto k_comb = k_combine_q<T, N>;
  smem_attr(kf_real, sm);
  smem_attr(kf_t, sm);
  smem_attr(ki_real, sm);
  smem_attr(kp_prod, 2 * sm);
  PlaneArgs pa{};
  pa.params = p->d_dummy_params;  // not read by these sources
  pa.g = f;
  pa.h = 2.0 * p->L / N;
  int launches = 0;
  // F = FFT(f)
  LBO_LAUNCH(p, "q_plane_fwd_f", s, kf_real, gp, blk, sm, pa, W1);
  Axis1Args ax{};
  LBO_LAUNCH(p, "q_axis1_fwd", s, ka_fwd, ga, blk, 0, ax, W1, FH);
  launches += 2;
  const int M = (int)qs->wm.size();
  const double pi = 3.141592653589793238462643383279502884;
  // hemisphere nodes in chunks of MB per launch (grid z): their inverse
  // transforms and products land in separate slots, summed in the order of m
  const int MB = q_chunk(B, M, N, generic_real_bytes(p->precision));
  cpx<T>* Wm1 = (cpx<T>*)(R2 + (size_t)B * n3);
  cpx<T>* Wm2 = Wm1 + (size_t)MB * B * H;
  T* Pm = (T*)(Wm2 + (size_t)MB * B * H);
  const double* dsig = qs->d_gsw + p->J;
  const double* dwm = dsig + 3 * M;
  const size_t total = (size_t)B * n3;
  const int cb = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
  // FP64 at N = 32: the per-(m) kernels with one thread per pencil
  // (quad_reg64.cuh) unless LBO_OPT_KERNEL = 2 asks for the shared-memory ones;
  // their phase factors come from a table after the chunk buffers
  constexpr bool R64 = std::is_same<T, double>::value && N == 32;
  const bool reg = R64 && p->kernel_choice != 2;
  cpx<double>* ptab = (cpx<double>*)(Pm + (size_t)MB * B * n3);
  if constexpr (R64) {
    if (reg) {
      LBO_LAUNCH(p, "q_phase_table", s, r64::k_q_phase_table_r64, p->J * M, 3 * N, 0, qs->d_gsw, dsig, M, pi,
                 2.0 * p->L, ptab);
      smem_attr(r64::k_plane_inv_prod_r64<4>, 2 * r64::PlaneR<4>::BYTES);
      launches += 1;
    }
  }
  for (int j = 0; j < p->J; ++j) {
    const double c = pi * p->gj[j] / (2.0 * p->L);
    for (int m0 = 0; m0 < M; m0 += MB) {
      const int mb = std::min(MB, M - m0);
      bool done = false;
      if constexpr (R64) {
        if (reg) {
          LBO_LAUNCH(p, "q_axis1_phase", s, r64::k_axis1_phase_r64, dim3(r64::RNC / 32, B, mb), 32, 0, FH, Wm1, Wm2,
                     ptab + (size_t)j * M * 3 * N, m0, (size_t)B * H);
          LBO_LAUNCH(p, "q_plane_inv_prod", s, r64::k_plane_inv_prod_r64<4>, dim3(N / 4, B, mb),
                     r64::PlaneR<4>::THREADS, 2 * r64::PlaneR<4>::BYTES, Wm1, Wm2, Pm, dwm, m0, (size_t)B * H,
                     total);
          done = true;
        }
      }
      if (!done) {
        LBO_LAUNCH(p, "q_axis1_phase", s, ka_ph, dim3(ga.x, B, mb), blk, 0, FH, Wm1, Wm2, dsig, m0, c,
                   (size_t)B * H);
        LBO_LAUNCH(p, "q_plane_inv_prod", s, kp_prod, dim3(gp.x, B, mb), blk, 2 * sm, Wm1, Wm2, Pm, dwm, m0,
                   (size_t)B * H, total);
      }
      LBO_LAUNCH(p, "q_sum_m", s, k_sum_m<T>, cb, 256, 0, Pm, Ps, mb, total, total, m0 == 0 ? 1 : 0);
      launches += 3;
    }
    pa.src = Ps;
    LBO_LAUNCH(p, "q_plane_fwd_p", s, kf_t, gp, blk, sm, pa, W1);
    Axis1Args a2{};
    a2.table = phi + (size_t)j * Q;
    a2.first = j == 0;
    LBO_LAUNCH(p, "q_axis1_fwd_acc", s, ka_acc, ga, blk, 0, a2, W1, QH);
    launches += 2;
  }
  LBO_LAUNCH(p, "q_axis1_inv", s, ka_inv, ga, blk, 0, ax, QH, QH);
  LBO_LAUNCH(p, "q_plane_inv", s, ki_real, gp, blk, sm, pa, QH, R1);
  // loss: f InvFFT(F omega), omega of Algorithm 1 (radial) or its hemisphere
  // quadrature, Eq. (2.16) (a multiplier per position)
  Axis1Args a3{};
  a3.table = omg3 ? (const void*)omg3 : (const void*)omg;
  LBO_LAUNCH(p, "q_plane_fwd_f", s, kf_real, gp, blk, sm, pa, W1);
  if (omg3) LBO_LAUNCH(p, "q_axis1_fwd_mul3_inv", s, ka_mult3, ga, blk, 0, a3, W1, W1);
  else LBO_LAUNCH(p, "q_axis1_fwd_mul_inv", s, ka_mult, ga, blk, 0, a3, W1, W1);
  LBO_LAUNCH(p, "q_plane_inv", s, ki_real, gp, blk, sm, pa, W1, R2);
  LBO_LAUNCH(p, "q_combine", s, k_comb, cb, 256, 0, f, R1, R2, out, total);
  launches += 6;
  if (p->mass_fix || p->moment_fix) {
    lbo_status st = launch_fixes(p, out, B, N, pa.h, s, &launches);
    if (st != LBO_OK) return st;
  }
  p->last_launches = launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "quadratic launch");
}

template <typename T>
static lbo_status dispatch_q(lbo_plan* p, QuadState* qs, const double* f, double* out, int B, const void* phi_v,
                      const void* omg_v, const void* omg3_v = nullptr) {
  const T *phi = (const T*)phi_v, *omg = (const T*)omg_v, *omg3 = (const T*)omg3_v;
  switch (p->N) {
    case 16: return run_quadratic<T, 16>(p, qs, f, out, B, phi, omg, omg3);
    case 24: return run_quadratic<T, 24>(p, qs, f, out, B, phi, omg, omg3);
    case 32: return run_quadratic<T, 32>(p, qs, f, out, B, phi, omg, omg3);
    case 48: return run_quadratic<T, 48>(p, qs, f, out, B, phi, omg, omg3);
    case 64: return run_quadratic<T, 64>(p, qs, f, out, B, phi, omg, omg3);
    default: return LBO_EUNSUPPORTED;
  }
}


// Q(f,f) in the two-fold precisions (lin_twofold.cu, lin_x2.cu); omg3: the
// Eq. (2.16) loss multiplier in the pair type, or null
lbo_status run_quadratic_twofold(lbo_plan* p, QuadState* qs, const double* f, double* out, int B,
                                 const void* omg3 = nullptr);

}  // namespace lbo

// The generic launch sequence of L[g] (plane and axis-1 kernels of
// lin_kernels.cuh), shared by the translation units that instantiate it for
// their transform precisions (lbo.cu: FP64 and FP32; lin_twofold.cu: the
// two-fold forms).  Each translation unit launches its own instances of the
// kernels, so each uploads its own FFT twiddle tables (upload_twiddles).
#pragma once
#include <cmath>
#include <type_traits>

#include "lbo_internal.h"
#include "lin_kernels.cuh"
#include "lin_reg64.cuh"

namespace lbo {

// Device tables of Algorithm 1 in the transform precision T.
template <typename T>
struct GenericTables {
  const T* phi;    // [J][3(N/2)^2+1] phi_j(|k|^2) / N^3
  const T* omega;  // [3(N/2)^2+1] omega(|k|^2) / N^3
  const T* phit;   // [J][N^3] phit_j, cyclic order
  const T* dct;    // [N/2+1][N/4] DCT-I coefficients of u^_j
};

// The plan's FP64 or FP32 tables (T = double or float).
template <typename T>
static GenericTables<T> plain_tables(const lbo_plan* p) {
  const bool f64 = sizeof(T) == 8;
  GenericTables<T> tb;
  tb.phi = (const T*)(f64 ? (const void*)p->d_phi64 : (const void*)p->d_phi32);
  tb.omega = (const T*)(f64 ? (const void*)p->d_omega64 : (const void*)p->d_omega32);
  tb.phit = (const T*)(f64 ? (const void*)p->d_phit64 : (const void*)p->d_phit32);
  tb.dct = (const T*)(f64 ? (const void*)p->d_dct64 : (const void*)p->d_dct32);
  return tb;
}

template <typename K>
static inline void set_smem(K kernel, size_t bytes) {
  raise_smem_limit((const void*)kernel, bytes);
}

template <int N>
struct PlanePPC { static constexpr int v = N == 16 ? 8 : (N == 32 ? 4 : (N == 24 ? 4 : (N == 48 ? 2 : 1))); };

// The launch sequence of L[g] on the generic kernels (Algorithm 1, in
// order): r^ = FFT(r); per radial node u^_j, psi_j = InvFFT(u^_j r^),
// M^h psi_j, psi^_j = FFT, L^+ += phi_j psi^_j; L+ = InvFFT(L^+); the loss
// term; the combination; the optional fixes.  ws: 3 half spectra + 3 real
// fields + the u^_j octant planes per instance, in T.
//
// Maxwellian cache (mc, may be null): u^_j of every radial node as whole
// octants ([J][B][(N/2+1)^3]) and the loss factor w = InvFFT(M^ omega)
// ([B][N^3]), computed by precompute_maxwellian_generic for these params;
// with it the u^_j DCTs and the transforms of w are not repeated.
template <typename T>
struct GenericCache {
  const T* uh;
  const T* w;
};

template <typename T, int N>
static lbo_status run_linearized_generic(lbo_plan* p, const GenericTables<T>& tb, const double* params,
                                         const double* g, double* out, int B, void* ws_raw,
                                         const GenericCache<T>* mc = nullptr) {
  constexpr int PPC = PlanePPC<N>::v, CW = 32, HC = N / 2 + 1;
  const size_t H = (size_t)N * N * HC, n3 = (size_t)N * N * N;
  cudaStream_t s = p->stream;
  unsigned char* ws = (unsigned char*)ws_raw;
  cpx<T>* RH = (cpx<T>*)ws;
  cpx<T>* W1 = RH + (size_t)B * H;
  cpx<T>* LH = W1 + (size_t)B * H;
  T* R1 = (T*)(LH + (size_t)B * H);
  T* R2 = R1 + (size_t)B * n3;
  T* R3 = R2 + (size_t)B * n3;
  T* UP = R3 + (size_t)B * n3;  // [B][HC]^3 u^_j after the axis-3 and axis-2 DCTs
  const T *dct = tb.dct, *phi = tb.phi, *omg = tb.omega, *phit = tb.phit;
  const int Q = 3 * (N / 2) * (N / 2) + 1;
  static_assert(PlaneSmem<T, N, PPC>::BYTES <= 227 * 1024, "plane kernels: shared memory of a block");
  static_assert(N * CW * sizeof(cpx<T>) + CW * HC * sizeof(T) <= 227 * 1024, "k_axis1: shared memory of a block");
  const size_t sm = PlaneSmem<T, N, PPC>::BYTES;
  const dim3 gp(N / PPC, B), ga((N * HC + CW - 1) / CW, B), blk(256);
  set_smem(k_plane_fwd<T, N, PPC, SRC_RATIO>, sm);
  set_smem(k_plane_fwd<T, N, PPC, SRC_REAL64>, sm);
  set_smem(k_plane_fwd<T, N, PPC, SRC_MAXW>, sm);
  set_smem(k_plane_inv<T, N, PPC, INV_MH_FWD>, sm);
  set_smem(k_plane_inv<T, N, PPC, INV_TO_REAL>, sm);
  PlaneArgs pa{};
  pa.params = params;
  pa.g = g;
  pa.h = 2.0 * p->L / N;
  pa.log_inv_eps = std::log(1.0 / p->eps);
  pa.cutoff = p->cutoff;
  auto kf_ratio = k_plane_fwd<T, N, PPC, SRC_RATIO>;
  auto kf_real = k_plane_fwd<T, N, PPC, SRC_REAL64>;
  auto kf_maxw = k_plane_fwd<T, N, PPC, SRC_MAXW>;
  auto ki_mh = k_plane_inv<T, N, PPC, INV_MH_FWD>;
  auto ki_real = k_plane_inv<T, N, PPC, INV_TO_REAL>;
  auto ka_fwd = k_axis1<T, N, CW, AX_FWD_STORE>;
  auto ka_mult = k_axis1<T, N, CW, AX_FWD_MULT_INV>;
  auto ka_acc = k_axis1<T, N, CW, AX_FWD_ACC>;
  auto ka_inv = k_axis1<T, N, CW, AX_INV_STORE>;
  auto ka_uhat = k_axis1<T, N, CW, AX_UHAT_INV>;
  auto ka_uhat_c = k_axis1<T, N, CW, AX_UHAT_CACHED>;
  constexpr int PL = UhatPlanes<N>::PL;  // octant planes per block
  auto k_up = k_uhat_planes<T, N, PL>;
  const size_t sm_up = sizeof(T) * ((size_t)PL * HC * HC + (size_t)HC * (N / 4));
  set_smem(k_up, sm_up);
  auto k_comb = k_combine<T, N>;
  // FP64 at N = 32: the gain loop's kernels with one thread per pencil
  // (lin_reg64.cuh) unless LBO_OPT_KERNEL = 2 asks for the shared-memory ones
  constexpr bool R64 = std::is_same<T, double>::value && N == 32;
  const bool reg = R64 && p->kernel_choice != 2;
  // cached: u^_j read whole from an octant (the cache, or, name
  // "axis1_uhat_octant_inv", the one uhat_finish completes for this call)
  auto launch_uhat = [&](const Axis1Args& a1, bool cached, const char* name = "axis1_uhat_cached_inv") {
    if constexpr (R64) {
      if (reg) {
        const dim3 gr(r64::RNC / 32, B);
        if (cached) LBO_LAUNCH(p, name, s, r64::k_axis1_uhat_r64<true>, gr, 32, 0, a1, RH, W1);
        else LBO_LAUNCH(p, "axis1_uhat_inv", s, r64::k_axis1_uhat_r64<false>, gr, 32, 0, a1, RH, W1);
        return;
      }
    }
    if (cached) LBO_LAUNCH(p, "axis1_uhat_cached_inv", s, ka_uhat_c, ga, blk, 0, a1, RH, W1);
    else LBO_LAUNCH(p, "axis1_uhat_inv", s, ka_uhat, ga, blk, 0, a1, RH, W1);
  };
  auto launch_mh = [&]() {
    if constexpr (R64) {
      if (reg) {
        // planes per CTA: LBO_OPT_PLANES (lbo_plan_autotune), default 4
        auto go = [&](auto rp) {
          constexpr int RP = decltype(rp)::value;
          auto k = r64::k_plane_mh_r64<RP>;
          set_smem(k, r64::PlaneR<RP>::BYTES);
          LBO_LAUNCH(p, "plane_inv_mh_fwd", s, k, dim3(N / RP, B), r64::PlaneR<RP>::THREADS, r64::PlaneR<RP>::BYTES,
                     (const double*)R2, W1);
        };
        if (p->r64_planes == 2) go(std::integral_constant<int, 2>());
        else if (p->r64_planes == 8) go(std::integral_constant<int, 8>());
        else go(std::integral_constant<int, 4>());
        return;
      }
    }
    LBO_LAUNCH(p, "plane_inv_mh_fwd", s, ki_mh, gp, blk, sm, pa, W1, (T*)nullptr);
  };
  auto launch_acc = [&](const Axis1Args& a2) {
    if constexpr (R64) {
      if (reg) {
        LBO_LAUNCH(p, "axis1_fwd_acc", s, r64::k_axis1_acc_r64, dim3(r64::RNC / 32, B), 32, 0, a2, W1, LH);
        return;
      }
    }
    LBO_LAUNCH(p, "axis1_fwd_acc", s, ka_acc, ga, blk, 0, a2, W1, LH);
  };
  int launches = 0;
  // r^ = FFT(r), r = g/M with the cut-off (Algorithm 1, gain term)
  LBO_LAUNCH(p, "plane_fwd_ratio", s, kf_ratio, gp, blk, sm, pa, W1);
  Axis1Args ax{};
  LBO_LAUNCH(p, "axis1_fwd", s, ka_fwd, ga, blk, 0, ax, W1, RH);
  launches += 2;
  const size_t HC3 = (size_t)HC * HC * HC;
  if constexpr (R64) {
    if (reg) {  // M^h / 2 for the register plane kernel, in R2 until the loss term
      LBO_LAUNCH(p, "mh_table", s, r64::k_mh_table_r64, B, 256, 0, params, pa.h, (double*)R2);
      launches += 1;
    }
  }
  for (int j = 0; j < p->J; ++j) {
    Axis1Args a1{};
    a1.dct = dct;
    a1.scale = 1.0 / (double)n3;
    if (mc) {
      // psi_j = InvFFT(u^_j r^), u^_j from the cache
      a1.uplanes = mc->uh + (size_t)j * B * HC3;
      launch_uhat(a1, true);
      launches -= 1;
    } else {
      a1.uplanes = UP;
      bool done = false;
      if constexpr (R64) {
        if (reg) {
          // u^_j on the whole octant (weight and the three DCT-I passes, one
          // block per instance), then psi_j reading it whole
          LBO_LAUNCH(p, "uhat_octant", s, r64::k_uhat_octant_r64, B, 320, 0, params, (const double*)phit + (size_t)j * n3,
                     pa.h, (double*)UP);
          launch_uhat(a1, true, "axis1_uhat_octant_inv");
          done = true;
        }
      }
      if (!done) {
        // u^_j = FFT(M^g phit_j), real and even: DCT-I of the octant, axes 3 and 2
        LBO_LAUNCH(p, "uhat_planes", s, k_up, dim3((HC + PL - 1) / PL, B), blk, sm_up, params,
                   phit + (size_t)j * n3, dct, pa.h, UP);
        // psi_j = InvFFT(u^_j r^), u^_j finished along axis 1 in the same kernel
        launch_uhat(a1, false);
      }
    }
    // psi_j <- M^h psi_j ; psi^_j = FFT(psi_j)
    launch_mh();
    // L^+ += phi_j psi^_j
    Axis1Args a2{};
    a2.table = phi + (size_t)j * Q;
    a2.first = j == 0;
    launch_acc(a2);
    launches += 4;
  }
  // L+ = InvFFT(L^+)
  LBO_LAUNCH(p, "axis1_inv", s, ka_inv, ga, blk, 0, ax, LH, LH);
  LBO_LAUNCH(p, "plane_inv", s, ki_real, gp, blk, sm, pa, LH, R1);
  // loss term: u = InvFFT(f^ omega), w = InvFFT(M^ omega)
  Axis1Args a3{};
  a3.table = omg;
  LBO_LAUNCH(p, "plane_fwd_g", s, kf_real, gp, blk, sm, pa, W1);
  LBO_LAUNCH(p, "axis1_fwd_mul_inv", s, ka_mult, ga, blk, 0, a3, W1, W1);
  LBO_LAUNCH(p, "plane_inv", s, ki_real, gp, blk, sm, pa, W1, R2);
  const T* ww = R3;
  if (mc) {
    ww = mc->w;
    launches -= 3;
  } else {
    LBO_LAUNCH(p, "plane_fwd_maxw", s, kf_maxw, gp, blk, sm, pa, W1);
    LBO_LAUNCH(p, "axis1_fwd_mul_inv", s, ka_mult, ga, blk, 0, a3, W1, W1);
    LBO_LAUNCH(p, "plane_inv", s, ki_real, gp, blk, sm, pa, W1, R3);
  }
  LBO_LAUNCH(p, "combine", s, k_comb, dim3(N, B), 256, 0, params, g, R1, R2, ww, out, pa.h, pa.log_inv_eps);
  launches += 9;
  if (p->mass_fix || p->moment_fix) {
    lbo_status st = launch_fixes(p, out, B, N, pa.h, s, &launches);
    if (st != LBO_OK) return st;
  }
  p->last_launches = launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "linearized launch");
  return LBO_OK;
}

// The Maxwellian-dependent factors of Algorithm 1 for the instances of
// params: u^_j = FFT(M^g phit_j) of every radial node as whole octants
// (k_uhat_planes for axes 3 and 2, k_uhat_finish for axis 1) into uh
// ([J][B][(N/2+1)^3]), and w = InvFFT(FFT(M) omega) into w ([B][N^3]).
// ws: the workspace of run_linearized_generic.
template <typename T, int N>
static lbo_status precompute_maxwellian_generic(lbo_plan* p, const GenericTables<T>& tb, const double* params,
                                                int B, void* ws_raw, T* uh, T* w) {
  constexpr int PPC = PlanePPC<N>::v, CW = 32, HC = N / 2 + 1;
  const size_t H = (size_t)N * N * HC, n3 = (size_t)N * N * N, HC3 = (size_t)HC * HC * HC;
  cudaStream_t s = p->stream;
  cpx<T>* W1 = (cpx<T>*)ws_raw + (size_t)B * H;
  const size_t sm = PlaneSmem<T, N, PPC>::BYTES;
  const dim3 gp(N / PPC, B), ga((N * HC + CW - 1) / CW, B), blk(256);
  set_smem(k_plane_fwd<T, N, PPC, SRC_MAXW>, sm);
  set_smem(k_plane_inv<T, N, PPC, INV_TO_REAL>, sm);
  constexpr int PL = UhatPlanes<N>::PL;
  auto k_up = k_uhat_planes<T, N, PL>;
  const size_t sm_up = sizeof(T) * ((size_t)PL * HC * HC + (size_t)HC * (N / 4));
  set_smem(k_up, sm_up);
  PlaneArgs pa{};
  pa.params = params;
  pa.h = 2.0 * p->L / N;
  pa.log_inv_eps = std::log(1.0 / p->eps);
  constexpr bool R64 = std::is_same<T, double>::value && N == 32;
  const bool reg = R64 && p->kernel_choice != 2;
  int per_j = 2;
  for (int j = 0; j < p->J; ++j) {
    T* dst = uh + (size_t)j * B * HC3;
    if constexpr (R64) {
      if (reg) {  // the octant kernel of the uncached register path: the same numbers
        LBO_LAUNCH(p, "cache_uhat_octant", s, r64::k_uhat_octant_r64, B, 320, 0, params,
                   (const double*)tb.phit + (size_t)j * n3, pa.h, (double*)dst);
        per_j = 1;
        continue;
      }
    }
    LBO_LAUNCH(p, "cache_uhat_planes", s, k_up, dim3((HC + PL - 1) / PL, B), blk, sm_up, params,
               tb.phit + (size_t)j * n3, tb.dct, pa.h, dst);
    LBO_LAUNCH(p, "cache_uhat_finish", s, (k_uhat_finish<T, N>), B, blk, 0, dst, tb.dct);
  }
  Axis1Args a3{};
  a3.table = tb.omega;
  LBO_LAUNCH(p, "cache_plane_fwd_maxw", s, (k_plane_fwd<T, N, PPC, SRC_MAXW>), gp, blk, sm, pa, W1);
  LBO_LAUNCH(p, "cache_axis1_fwd_mul_inv", s, (k_axis1<T, N, CW, AX_FWD_MULT_INV>), ga, blk, 0, a3, W1, W1);
  LBO_LAUNCH(p, "cache_plane_inv", s, (k_plane_inv<T, N, PPC, INV_TO_REAL>), gp, blk, sm, pa, W1, w);
  p->last_launches = per_j * p->J + 3;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "Maxwellian cache launch");
}

template <typename T>
static lbo_status dispatch_generic(lbo_plan* p, const GenericTables<T>& tb, const double* params, const double* g,
                                  double* out, int B, void* ws, const GenericCache<T>* mc = nullptr) {
  switch (p->N) {
    case 16: return run_linearized_generic<T, 16>(p, tb, params, g, out, B, ws, mc);
    case 24: return run_linearized_generic<T, 24>(p, tb, params, g, out, B, ws, mc);
    case 32: return run_linearized_generic<T, 32>(p, tb, params, g, out, B, ws, mc);
    case 48: return run_linearized_generic<T, 48>(p, tb, params, g, out, B, ws, mc);
    case 64: return run_linearized_generic<T, 64>(p, tb, params, g, out, B, ws, mc);
    default: return LBO_EUNSUPPORTED;
  }
}

template <typename T>
static lbo_status dispatch_precompute(lbo_plan* p, const GenericTables<T>& tb, const double* params, int B, void* ws,
                                      void* uh, void* w) {
  switch (p->N) {
    case 16: return precompute_maxwellian_generic<T, 16>(p, tb, params, B, ws, (T*)uh, (T*)w);
    case 24: return precompute_maxwellian_generic<T, 24>(p, tb, params, B, ws, (T*)uh, (T*)w);
    case 32: return precompute_maxwellian_generic<T, 32>(p, tb, params, B, ws, (T*)uh, (T*)w);
    case 48: return precompute_maxwellian_generic<T, 48>(p, tb, params, B, ws, (T*)uh, (T*)w);
    case 64: return precompute_maxwellian_generic<T, 64>(p, tb, params, B, ws, (T*)uh, (T*)w);
    default: return LBO_EUNSUPPORTED;
  }
}

}  // namespace lbo

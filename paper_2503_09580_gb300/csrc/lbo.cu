// liblbo: C ABI (include/lbo.h) of the GB300 fast Fourier spectral
// linearized Boltzmann collision operator.  Plan management, the tables of
// Algorithm 1 (its precomputation step) and the launch sequence of the
// generic FP64 / FP32 path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbo.h"
#include "lbo_internal.h"
#include "lin_generic.cuh"

namespace lbo {
static thread_local std::string g_last_error;

lbo_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return LBO_ECUDA;
}

void set_error_text(const char* msg) { g_last_error = msg; }

// ------------------------------------------------------------ quadrature
// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on the
// three-term recurrence of the Legendre polynomials.
void gauss_legendre(int J, std::vector<double>& x, std::vector<double>& w) {
  x.assign(J, 0.0);
  w.assign(J, 0.0);
  for (int i = 0; i < (J + 1) / 2; ++i) {
    long double z = std::cos(3.14159265358979323846264338327950288L * (i + 0.75L) / (J + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= J; ++k) {
        long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (J == 1) { p1 = z; p0 = 1; }
      dp = J * (z * p1 - p0) / (z * z - 1);
      long double dz = p1 / dp;
      z -= dz;
      if (std::fabs((double)dz) < 1e-19) break;
    }
    // recompute derivative at the converged node
    long double p0 = 1, p1 = z;
    for (int k = 2; k <= J; ++k) {
      long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = J * (z * p1 - p0) / (z * z - 1);
    long double wt = 2.0L / ((1 - z * z) * dp * dp);
    x[i] = (double)(-z);
    x[J - 1 - i] = (double)z;
    w[i] = w[J - 1 - i] = (double)wt;
  }
}

static double sinc_h(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

}  // namespace lbo

using namespace lbo;

// ------------------------------------------------------------------ plan
static lbo_status ensure_twiddles() {
  cudaError_t e = upload_twiddles();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "twiddle upload");
}

static int qmax_of(int N) { return 3 * (N / 2) * (N / 2) + 1; }

template <typename T, int N>
static lbo_status build_phit(lbo_plan* p, const double* d_stab, T* d_phit);

static void free_tables(lbo_plan* p) {
  free_twofold_tables(p);
  void* ptrs[] = {p->d_phi64, p->d_omega64, p->d_phit64, p->d_phi32, p->d_omega32, p->d_phit32, p->d_dummy_params,
                  p->d_dct64, p->d_dct32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->d_phi64 = p->d_omega64 = p->d_phit64 = nullptr;
  p->d_phi32 = p->d_omega32 = p->d_phit32 = nullptr;
  p->d_dct64 = nullptr;
  p->d_dct32 = nullptr;
  p->d_dummy_params = nullptr;
}

static lbo_status build_tables(lbo_plan* p) {
  lbo_status st = ensure_twiddles();
  if (st != LBO_OK) return st;
  free_tables(p);
  const int N = p->N, J = p->J, Q = qmax_of(N);
  std::vector<double> x, w;
  gauss_legendre(J, x, w);
  p->gj.resize(J);
  p->wj.resize(J);
  p->Bj.resize(J);
  for (int j = 0; j < J; ++j) {
    double g = 0.5 * p->R * (x[j] + 1.0);
    p->gj[j] = g;
    p->wj[j] = 0.5 * p->R * w[j] * g * g;              // folds g^2 of Eq. (2.13)
    p->Bj[j] = p->C * std::pow(g, 2.0 * (1.0 - p->omega));  // Eq. (2.4)
  }
  const double inv_n3 = 1.0 / ((double)N * N * N);
  const double pi = 3.141592653589793238462643383279502884;
  std::vector<double> stab((size_t)J * Q), phi((size_t)J * Q), om(Q, 0.0);
  for (int q = 0; q < Q; ++q) {
    double kn = std::sqrt((double)q);
    for (int j = 0; j < J; ++j) {
      double s = sinc_h(pi * p->gj[j] * kn / (2.0 * p->L));
      stab[(size_t)j * Q + q] = s * inv_n3;
      // phi_{j,k} = 4 pi^2 w_j B(g_j) s_{j,k}: the constant of Algorithm 1
      // re-derived from Eqs. (3.5)-(3.8) (the printed 32 pi^2 breaks L[M] = 0)
      phi[(size_t)j * Q + q] = 4.0 * pi * pi * p->wj[j] * p->Bj[j] * s * inv_n3;
      om[q] += p->wj[j] * p->Bj[j] * sinc_h(pi * p->gj[j] * kn / p->L);
    }
    om[q] *= 16.0 * pi * pi * inv_n3;  // omega_k of Algorithm 1
  }
  cudaError_t e;
  const size_t n3 = (size_t)N * N * N;
  double* d_stab = nullptr;
#define TRY(x)                                  \
  do {                                          \
    e = (x);                                    \
    if (e != cudaSuccess) {                     \
      if (d_stab) cudaFree(d_stab);             \
      free_tables(p);                           \
      return cuda_fail(e, #x);                  \
    }                                           \
  } while (0)
  TRY(cudaMalloc(&p->d_phi64, sizeof(double) * J * Q));
  TRY(cudaMalloc(&p->d_omega64, sizeof(double) * Q));
  TRY(cudaMalloc(&p->d_phit64, sizeof(double) * J * n3));
  TRY(cudaMalloc(&p->d_phi32, sizeof(float) * J * Q));
  TRY(cudaMalloc(&p->d_omega32, sizeof(float) * Q));
  TRY(cudaMalloc(&p->d_phit32, sizeof(float) * J * n3));
  TRY(cudaMalloc(&p->d_dummy_params, sizeof(double) * 5 * std::max(J, 1)));
  TRY(cudaMalloc(&d_stab, sizeof(double) * J * Q));
  TRY(cudaMemcpy(p->d_phi64, phi.data(), sizeof(double) * J * Q, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(p->d_omega64, om.data(), sizeof(double) * Q, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(d_stab, stab.data(), sizeof(double) * J * Q, cudaMemcpyHostToDevice));
  TRY(cudaMemset(p->d_dummy_params, 0, sizeof(double) * 5 * std::max(J, 1)));
  {
    std::vector<float> f((size_t)J * Q);
    for (size_t i = 0; i < f.size(); ++i) f[i] = (float)phi[i];
    TRY(cudaMemcpy(p->d_phi32, f.data(), sizeof(float) * J * Q, cudaMemcpyHostToDevice));
    std::vector<float> fo(Q);
    for (int i = 0; i < Q; ++i) fo[i] = (float)om[i];
    TRY(cudaMemcpy(p->d_omega32, fo.data(), sizeof(float) * Q, cudaMemcpyHostToDevice));
  }
  {
    // c_d cos(2 pi k d / N), k = 0..N/2, d = 0..N/4-1 (c_0 = 1, c_d = 2);
    // the cosines are the correctly rounded ones of the twiddle tables (N
    // divides 64 or 48), so zeros are exact and the register kernels'
    // compile-time cosines (cos32) are the same numbers
    const int HN = N / 2 + 1, Q4 = N / 4;
    std::vector<double> dc((size_t)HN * Q4);
    std::vector<float> df(dc.size());
    for (int k = 0; k < HN; ++k)
      for (int d = 0; d < Q4; ++d) {
        const double c = 64 % N == 0 ? kTw64Hi[(k * d * (64 / N)) % 64][0] : kTw48Hi[(k * d * (48 / N)) % 48][0];
        dc[(size_t)k * Q4 + d] = (d == 0 ? 1.0 : 2.0) * c;
        df[(size_t)k * Q4 + d] = (float)dc[(size_t)k * Q4 + d];
      }
    TRY(cudaMalloc(&p->d_dct64, sizeof(double) * dc.size()));
    TRY(cudaMalloc(&p->d_dct32, sizeof(float) * df.size()));
    TRY(cudaMemcpy(p->d_dct64, dc.data(), sizeof(double) * dc.size(), cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(p->d_dct32, df.data(), sizeof(float) * df.size(), cudaMemcpyHostToDevice));
  }
#undef TRY
  lbo_status s2;
  switch (N) {
    case 16: s2 = build_phit<double, 16>(p, d_stab, p->d_phit64); break;
    case 24: s2 = build_phit<double, 24>(p, d_stab, p->d_phit64); break;
    case 32: s2 = build_phit<double, 32>(p, d_stab, p->d_phit64); break;
    case 48: s2 = build_phit<double, 48>(p, d_stab, p->d_phit64); break;
    case 64: s2 = build_phit<double, 64>(p, d_stab, p->d_phit64); break;
    default: s2 = LBO_EUNSUPPORTED;
  }
  cudaFree(d_stab);
  if (s2 != LBO_OK) {
    free_tables(p);
    return s2;
  }
  p->tables_dirty = false;
  p->mc_valid = false;
  return LBO_OK;
}

// ------------------------------------------------------------ workspace
static lbo_status ensure_ws_bytes(lbo_plan* p, size_t bytes) {
  if (p->ws && bytes <= p->ws_bytes) return LBO_OK;
  if (p->ws) {
    cudaFree(p->ws);
    p->ws = nullptr;
    p->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&p->ws, bytes);
  if (e != cudaSuccess) {
    p->ws = nullptr;
    cudaGetLastError();
    g_last_error = "workspace allocation";
    return LBO_ENOMEM;
  }
  p->ws_bytes = bytes;
  return LBO_OK;
}

static lbo_status ensure_workspace(lbo_plan* p, int batch) {
  const size_t N = p->N, H = N * N * (N / 2 + 1), n3 = N * N * N, HN = N / 2 + 1;
  // generic path: 3 half spectra + 3 real fields + the u^_j DCT planes per
  // instance, sized for FP64 (for the FP64 pairs: twice that)
  const size_t rb = generic_real_bytes(p->precision);
  return ensure_ws_bytes(p, (size_t)batch * (3 * H * 2 * rb + 3 * n3 * rb + HN * HN * HN * rb));
}

static lbo_status ensure_stage(lbo_plan* p, size_t in_doubles, size_t out_doubles, size_t par_doubles) {
  auto grow = [&](double*& ptr, size_t& cap, size_t need) -> lbo_status {
    if (need <= cap) return LBO_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    if (cudaMalloc(&ptr, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      g_last_error = "staging allocation";
      return LBO_ENOMEM;
    }
    cap = need;
    return LBO_OK;
  };
  lbo_status s = grow(p->stage_in, p->stage_in_cap, in_doubles);
  if (s == LBO_OK) s = grow(p->stage_out, p->stage_out_cap, out_doubles);
  if (s == LBO_OK) s = grow(p->stage_par, p->stage_par_cap, par_doubles);
  return s;
}

// phit_j = IDFT(s_j) for all j, FP64, then an FP32 copy.
template <typename T, int N>
__global__ void k_fill_spectrum(const double* __restrict__ stab, cpx<double>* __restrict__ dst, int Q) {
  constexpr int HC = N / 2 + 1, NC = N * HC;
  const int j = blockIdx.y;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * NC; t += gridDim.x * blockDim.x) {
    int r = t / NC, col = t % NC, p2 = col / HC, k3 = col % HC;
    int k1 = centred<N>(freq_of_pos<N>(r)), k2 = centred<N>(freq_of_pos<N>(p2));
    dst[(size_t)j * N * NC + t] = make_c(stab[(size_t)j * Q + k1 * k1 + k2 * k2 + k3 * k3], 0.0);
  }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

template <typename T, int N>
static lbo_status build_phit(lbo_plan* p, const double* d_stab, T* d_phit) {
  constexpr int PPC = PlanePPC<N>::v, CW = 32;
  const int J = p->J, Q = qmax_of(N);
  const size_t H = (size_t)N * N * (N / 2 + 1), n3 = (size_t)N * N * N;
  cpx<double>* spec = nullptr;
  cudaError_t e = cudaMalloc(&spec, sizeof(cpx<double>) * H * J);
  if (e != cudaSuccess) return cuda_fail(e, "phit spectrum");
  k_fill_spectrum<double, N><<<dim3(64, J), 256>>>(d_stab, spec, Q);
  Axis1Args ax{};
  k_axis1<double, N, CW, AX_INV_STORE><<<dim3((N * (N / 2 + 1) + CW - 1) / CW, J), 256>>>(ax, spec, spec);
  PlaneArgs pa{};
  pa.params = p->d_dummy_params;
  pa.h = 2.0 * p->L / N;
  size_t sm = PlaneSmem<double, N, PPC>::BYTES;
  set_smem(k_plane_inv<double, N, PPC, INV_TO_REAL>, sm);
  k_plane_inv<double, N, PPC, INV_TO_REAL><<<dim3(N / PPC, J), 256, sm>>>(pa, spec, (double*)p->d_phit64);
  k_to_float<<<256, 256>>>((const double*)p->d_phit64, (float*)p->d_phit32, (size_t)J * n3);
  e = cudaDeviceSynchronize();
  cudaFree(spec);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "phit build");
  (void)d_phit;
  return LBO_OK;
}

template <typename T>
static lbo_status dispatch_lin(lbo_plan* p, const double* params, const double* g, double* out, int B,
                               const void* cuh, const void* cw) {
  GenericCache<T> mc{(const T*)cuh, (const T*)cw};
  return dispatch_generic<T>(p, plain_tables<T>(p), params, g, out, B, p->ws, cuh ? &mc : nullptr);
}

// kernel set of an apply call: 1 the fused FP32 kernels (N = 32), 0 generic
static int kernel_path(const lbo_plan* p) {
  return p->precision == LBO_PREC_FP32 && p->N == 32 && p->kernel_choice == 0 ? 1 : 0;
}

// bytes of one real number of the generic path's transform arithmetic
static size_t transform_real_bytes(int prec) {
  return prec == LBO_PREC_FP32 || is_split16_precision(prec) ? 4 : (prec == LBO_PREC_FP64X2 ? 16 : 8);
}

static lbo_status grow_buffer(void*& ptr, size_t& cap, size_t need, const char* what) {
  if (need <= cap) return LBO_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  if (cudaMalloc(&ptr, need) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = what;
    return LBO_ENOMEM;
  }
  cap = need;
  return LBO_OK;
}

static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------ ABI
extern "C" {

const char* lbo_status_string(lbo_status s) {
  switch (s) {
    case LBO_OK: return "ok";
    case LBO_EINVAL: return "invalid argument";
    case LBO_ENOMEM: return "out of memory";
    case LBO_ECUDA: return "CUDA error";
    case LBO_ENOTCONV: return "not converged";
    case LBO_EBREAKDOWN: return "Krylov breakdown";
    case LBO_ENAN: return "non-finite value";
    case LBO_EUNSUPPORTED: return "unsupported configuration";
    case LBO_ETIMEOUT: return "a kernel's bounded wait ran out";
  }
  return "unknown status";
}

const char* lbo_last_error(void) { return g_last_error.c_str(); }

lbo_status lbo_plan_create(int N, double box, double vhs_omega, int radial_nodes, lbo_plan** out) {
  if (!out) return LBO_EINVAL;
  *out = nullptr;
  if (N != 16 && N != 24 && N != 32 && N != 48 && N != 64) return LBO_EUNSUPPORTED;
  if (!(box > 0.0) || !(vhs_omega >= 0.5 && vhs_omega <= 1.0) || radial_nodes < 1 || radial_nodes > 256)
    return LBO_EINVAL;
  lbo_plan* p = new lbo_plan();
  p->N = N;
  p->L = box;
  p->omega = vhs_omega;
  p->J = radial_nodes;
  p->R = 4.0 * box / (3.0 + std::sqrt(2.0));
  p->C = 1.0 / (4.0 * 3.141592653589793238462643383279502884);
  p->eps = 1e-9;
  p->cutoff = 1;
  p->hemi_p = 4;
  p->precision = LBO_PREC_FP64;
  cudaGetDevice(&p->device);
  lbo_status st = build_tables(p);
  if (st != LBO_OK) {
    lbo_plan_destroy(p);
    return st;
  }
  *out = p;
  return LBO_OK;
}

lbo_status lbo_plan_set(lbo_plan* p, lbo_option key, double v) {
  if (!p) return LBO_EINVAL;
  switch (key) {
    case LBO_OPT_R:
      if (!(v > 0.0)) return LBO_EINVAL;
      p->R = v;
      p->tables_dirty = true;
      break;
    case LBO_OPT_C:
      if (!(v > 0.0)) return LBO_EINVAL;
      p->C = v;
      p->tables_dirty = true;
      break;
    case LBO_OPT_EPS:
      if (!(v > 0.0 && v < 1.0)) return LBO_EINVAL;
      p->eps = v;
      break;
    case LBO_OPT_CUTOFF: p->cutoff = v != 0.0; break;
    case LBO_OPT_MASS_FIX: p->mass_fix = v != 0.0; break;
    case LBO_OPT_MOMENT_FIX: p->moment_fix = v != 0.0; break;
    case LBO_OPT_HEMISPHERE_P:
      if (!(v >= 1.0 && v <= 32.0)) return LBO_EINVAL;
      p->hemi_p = (int)v;
      break;
    case LBO_OPT_PRECISION:
      if (!(v == 0.0 || v == 1.0 || v == 2.0 || v == 3.0 || v == 4.0 || v == 5.0)) return LBO_EINVAL;
      p->precision = (int)v;
      break;
    case LBO_OPT_KERNEL:
      if (v != 0.0 && v != 1.0 && v != 2.0) return LBO_EINVAL;
      p->kernel_choice = (int)v;
      break;
    case LBO_OPT_JGROUPS:
      if (!(v >= 0.0 && v <= 64.0)) return LBO_EINVAL;
      p->jgroups = (int)v;
      break;
    case LBO_OPT_Q_SINC_QUADRATURE:
      if (v != 0.0 && v != 1.0) return LBO_EINVAL;
      p->q_sinc_quad = (int)v;
      break;
    case LBO_OPT_PLANES:
      if (v != 0.0 && v != 2.0 && v != 4.0 && v != 8.0) return LBO_EINVAL;
      p->r64_planes = (int)v;
      break;
    default: return LBO_EINVAL;
  }
  return LBO_OK;
}

lbo_status lbo_plan_set_stream(lbo_plan* p, void* stream) {
  if (!p) return LBO_EINVAL;
  p->stream = (cudaStream_t)stream;
  return LBO_OK;
}

lbo_status lbo_apply_linearized(lbo_plan* p, const double* params, const double* g, double* out, int batch) {
  if (!p || batch < 0) return LBO_EINVAL;
  if (batch == 0) {
    p->last_launches = 0;
    return LBO_OK;
  }
  if (!params || !g || !out || out == g) return LBO_EINVAL;
  if (p->tables_dirty) {
    lbo_status st = build_tables(p);
    if (st != LBO_OK) return st;
  }
  lbo_status st = ensure_workspace(p, batch);
  if (st != LBO_OK) return st;
  const size_t n3 = (size_t)p->N * p->N * p->N;
  const bool dev = is_device_ptr(params) && is_device_ptr(g) && is_device_ptr(out);
  const double *dp = params, *dg = g;
  double* dout = out;
  if (!dev) {
    st = ensure_stage(p, (size_t)batch * n3, (size_t)batch * n3, (size_t)batch * 5);
    if (st != LBO_OK) return st;
    cudaError_t e = cudaMemcpyAsync(p->stage_par, params, sizeof(double) * 5 * batch, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->stage_in, g, sizeof(double) * n3 * batch, cudaMemcpyDefault, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    dp = p->stage_par;
    dg = p->stage_in;
    dout = p->stage_out;
  }
  // the Maxwellian cache, if it was made for exactly this call's Maxwellians
  const int path = kernel_path(p);
  const bool cached = p->mc_valid && p->mc_params == dp && p->mc_batch == batch && p->mc_precision == p->precision &&
                      p->mc_path == path;
  const void* cuh = cached ? p->mc_uh : nullptr;
  const void* cw = cached ? p->mc_w : nullptr;
  if (path == 1) {
    int G = p->jgroups > 0 ? std::min(p->jgroups, p->J) : std::min(fused32_default_groups(batch), p->J);
    st = ensure_ws_bytes(p, fused32_workspace_bytes(batch, G, p->J));
    if (st != LBO_OK) return st;
    int launches = 0;
    st = run_linearized_fused32(p, dp, dg, dout, batch, p->ws, G, &launches, (const float*)cuh);
    if (st == LBO_OK && (p->mass_fix || p->moment_fix))
      st = launch_fixes(p, dout, batch, p->N, 2.0 * p->L / p->N, p->stream, &launches);
    p->last_launches = launches;
  } else if (is_twofold_precision(p->precision)) {
    st = run_linearized_twofold(p, dp, dg, dout, batch, cuh, cw);
  } else if (is_split16_precision(p->precision)) {
    if (!dftmm_supported(p->N)) {
      g_last_error = "split 16-bit tensor-core precisions: N = 16, 32 or 64";
      return LBO_EUNSUPPORTED;
    }
    p->last_launches = 0;
    const size_t HC = p->N / 2 + 1, n3 = (size_t)p->N * p->N * p->N;
    if (!cached) {
      // u^_j and w for this call, by the generic FP32 kernels
      const size_t uh_bytes = (size_t)p->J * batch * HC * HC * HC * 4;
      st = grow_buffer(p->tc_scratch, p->tc_scratch_bytes, uh_bytes + (size_t)batch * n3 * 4,
                       "tensor-core scratch allocation");
      if (st != LBO_OK) return st;
      cuh = p->tc_scratch;
      cw = (unsigned char*)p->tc_scratch + uh_bytes;
      st = dispatch_precompute<float>(p, plain_tables<float>(p), dp, batch, p->ws, (void*)cuh, (void*)cw);
      if (st != LBO_OK) return st;
    }
    st = run_linearized_dftmm(p, dp, dg, dout, batch, (const float*)cuh, (const float*)cw, p->ws);
    if (st == LBO_OK && (p->mass_fix || p->moment_fix)) {
      int launches = p->last_launches;
      st = launch_fixes(p, dout, batch, p->N, 2.0 * p->L / p->N, p->stream, &launches);
      p->last_launches = launches;
    }
  } else {
    st = p->precision == LBO_PREC_FP64 ? dispatch_lin<double>(p, dp, dg, dout, batch, cuh, cw)
                                       : dispatch_lin<float>(p, dp, dg, dout, batch, cuh, cw);
  }
  if (st != LBO_OK) return st;
  if (!dev) {
    cudaError_t e = cudaMemcpyAsync(out, p->stage_out, sizeof(double) * n3 * batch, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
    if (is_split16_precision(p->precision)) return dftmm_check(p);
  }
  return LBO_OK;
}

lbo_status lbo_plan_cache_maxwellians(lbo_plan* p, const double* params, int batch) {
  if (!p || batch < 0) return LBO_EINVAL;
  p->mc_valid = false;
  if (!params || batch == 0) return LBO_OK;  // dropped; the buffers are kept for reuse
  if (!is_device_ptr(params)) {
    set_error_text("Maxwellian cache: params must be a device pointer");
    return LBO_EINVAL;
  }
  if (p->tables_dirty) {
    lbo_status st = build_tables(p);
    if (st != LBO_OK) return st;
  }
  const int path = kernel_path(p);
  const size_t N = p->N, HC = N / 2 + 1, n3 = N * N * N;
  const size_t rb = transform_real_bytes(p->precision);
  const size_t uh_bytes = path == 1 ? fused32_uhat_bytes(batch, p->J) : (size_t)p->J * batch * HC * HC * HC * rb;
  const size_t w_bytes = path == 1 ? 0 : (size_t)batch * n3 * rb;
  auto grow = [&](void*& ptr, size_t& cap, size_t need) -> lbo_status {
    if (need <= cap) return LBO_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    if (cudaMalloc(&ptr, need) != cudaSuccess) {
      cudaGetLastError();
      set_error_text("Maxwellian cache allocation");
      return LBO_ENOMEM;
    }
    cap = need;
    return LBO_OK;
  };
  lbo_status st = grow(p->mc_uh, p->mc_uh_bytes, uh_bytes);
  if (st == LBO_OK && w_bytes) st = grow(p->mc_w, p->mc_w_bytes, w_bytes);
  if (st == LBO_OK && path == 0) st = ensure_workspace(p, batch);
  if (st != LBO_OK) return st;
  if (path == 1) st = precompute_fused32(p, params, batch, (float*)p->mc_uh);
  else if (is_twofold_precision(p->precision)) st = precompute_twofold(p, params, batch, p->mc_uh, p->mc_w);
  else if (p->precision == LBO_PREC_FP64)
    st = dispatch_precompute<double>(p, plain_tables<double>(p), params, batch, p->ws, p->mc_uh, p->mc_w);
  else st = dispatch_precompute<float>(p, plain_tables<float>(p), params, batch, p->ws, p->mc_uh, p->mc_w);
  if (st != LBO_OK) return st;
  p->mc_params = params;
  p->mc_batch = batch;
  p->mc_precision = p->precision;
  p->mc_path = path;
  p->mc_valid = true;
  return LBO_OK;
}

lbo_status lbo_apply_quadratic(lbo_plan* p, const double* f, double* out, int batch) {
  if (!p || batch < 0) return LBO_EINVAL;
  if (batch == 0) {
    p->last_launches = 0;
    return LBO_OK;
  }
  if (!f || !out || out == f) return LBO_EINVAL;
  if (p->tables_dirty) {
    lbo_status st = build_tables(p);
    if (st != LBO_OK) return st;
  }
  const size_t n3 = (size_t)p->N * p->N * p->N;
  const bool dev = is_device_ptr(f) && is_device_ptr(out);
  const double* df = f;
  double* dout = out;
  lbo_status st;
  if (!dev) {
    st = ensure_stage(p, (size_t)batch * n3, (size_t)batch * n3, 5);
    if (st != LBO_OK) return st;
    cudaError_t e = cudaMemcpyAsync(p->stage_in, f, sizeof(double) * n3 * batch, cudaMemcpyDefault, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    df = p->stage_in;
    dout = p->stage_out;
  }
  st = apply_quadratic_device(p, df, dout, batch);
  if (st != LBO_OK) return st;
  if (!dev) {
    cudaError_t e = cudaMemcpyAsync(out, p->stage_out, sizeof(double) * n3 * batch, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  }
  return LBO_OK;
}

lbo_status lbo_plan_sync(lbo_plan* p) {
  if (!p) return LBO_EINVAL;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  return dftmm_check(p);  // a tensor-core pass that gave up waiting
}

int lbo_plan_last_launches(const lbo_plan* p) { return p ? p->last_launches : 0; }

void lbo_plan_destroy(lbo_plan* p) {
  if (!p) return;
  free_tables(p);
  if (p->mc_uh) cudaFree(p->mc_uh);
  if (p->mc_w) cudaFree(p->mc_w);
  if (p->tc_scratch) cudaFree(p->tc_scratch);
  if (p->blk_red) cudaFree(p->blk_red);
  free_dftmm(p);
  if (p->ws) cudaFree(p->ws);
  if (p->stage_in) cudaFree(p->stage_in);
  if (p->stage_out) cudaFree(p->stage_out);
  if (p->stage_par) cudaFree(p->stage_par);
  free_quadratic(p);
  free_profile(p);
  delete p;
}

}  // extern "C"

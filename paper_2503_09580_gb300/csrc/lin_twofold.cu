// L[g] in the two-fold precisions (twofold.cuh): LBO_PREC_FP32X2, pairs of
// FP32 numbers on the FP32 pipe (about 48 significant bits), and
// LBO_PREC_FP64X2, pairs of FP64 numbers (about 106 bits).  The generic
// kernel sequence of Algorithm 1 (lin_generic.cuh) runs with every transform
// and every product of the gain and loss terms in the two-fold type; the
// Maxwellians, the ratio r = g/M and the cut-off stay FP64 as in the other
// forms, and so do the inputs, the outputs and the final combination.
//
// Tables: the FFT twiddles and the DCT-I coefficients of u^_j come from the
// double-pair table twiddles_hi.h (accurate to ~2^-106); phi_j, omega and
// phit_j are the plan's FP64 tables carried over (split into a float pair,
// or with a zero low part).  Their FP64 rounding is a pointwise relative
// perturbation of the multipliers and of u_j, which the convolution does not
// amplify; what the two-fold arithmetic removes is the rounding of the
// transforms themselves, whose error grows with max|r| (Sec. 3.3).  The
// two-fold tables are built on the first call in such a precision and kept
// until the plan's tables are rebuilt.
#include <cuda_runtime.h>

#include <vector>

#include "lin_generic.cuh"
#include "quad_generic.cuh"

namespace lbo {

// defined in lin_x2.cu, one translation unit per (pair type, N)
#define LBO_X2_DECL(b, n)                                                                                       \
  lbo_status x2_lin_##b##_##n(lbo_plan* p, const void* const* tb, const double* params, const double* g,      \
                              double* out, int B, const void* cuh, const void* cw);                          \
  lbo_status x2_cache_##b##_##n(lbo_plan* p, const void* const* tb, const double* params, int B, void* uh,      \
                                void* w);                                                                    \
  lbo_status x2_quad_##b##_##n(lbo_plan* p, QuadState* qs, const void* const* tb, const double* f, double* out, \
                               int B, const void* omg3);
LBO_X2_DECL(1, 16)
LBO_X2_DECL(1, 24)
LBO_X2_DECL(1, 32)
LBO_X2_DECL(1, 48)
LBO_X2_DECL(1, 64)
LBO_X2_DECL(2, 16)
LBO_X2_DECL(2, 32)
#undef LBO_X2_DECL

namespace {

__global__ void k_split_f32x2(const double* __restrict__ a, f32x2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = f32x2(a[i]);
}

__global__ void k_widen_f64x2(const double* __restrict__ a, f64x2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = f64x2(a[i], 0.0);
}

// cos(2 pi t / N) as a double pair from the twiddle table
void cos_pair(int N, long t, double* hi, double* lo) {
  if (64 % N == 0) {
    const int m = (int)(((64 / N) * t) % 64);
    *hi = kTw64Hi[m][0];
    *lo = kTw64Hi[m][1];
  } else {
    const int m = (int)(((48 / N) * t) % 48);
    *hi = kTw48Hi[m][0];
    *lo = kTw48Hi[m][1];
  }
}

template <typename T>
lbo_status upload(const std::vector<T>& h, void** d) {
  cudaError_t e = cudaMalloc(d, sizeof(T) * h.size());
  if (e == cudaSuccess) e = cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (*d) cudaFree(*d);
    *d = nullptr;
    return cuda_fail(e, "two-fold tables");
  }
  return LBO_OK;
}

// Tables of precision `prec` (FP32X2 or FP64X2); built once.
template <typename T>
lbo_status build(lbo_plan* p, void** slot) {
  if (slot[0]) return LBO_OK;
  const int N = p->N, J = p->J, Q = 3 * (N / 2) * (N / 2) + 1, HN = N / 2 + 1, Q4 = N / 4;
  const size_t n3 = (size_t)N * N * N;
  std::vector<double> phi((size_t)J * Q), om(Q);
  cudaError_t e = cudaMemcpy(phi.data(), p->d_phi64, sizeof(double) * phi.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(om.data(), p->d_omega64, sizeof(double) * Q, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "two-fold tables: read back");
  std::vector<T> hphi(phi.size()), hom(Q), hdct((size_t)HN * Q4);
  for (size_t i = 0; i < phi.size(); ++i) hphi[i] = T(phi[i]);
  for (int i = 0; i < Q; ++i) hom[i] = T(om[i]);
  for (int k = 0; k < HN; ++k)
    for (int d = 0; d < Q4; ++d) {
      double hi, lo;
      cos_pair(N, (long)k * d, &hi, &lo);
      const double c = d == 0 ? 1.0 : 2.0;  // c_d of the DCT-I (exact scaling)
      if constexpr (sizeof(T) == 16) {
        hdct[(size_t)k * Q4 + d] = T(c * hi, c * lo);
      } else {
        float fh, fl;
        split_to_float_pair(c * hi, c * lo, &fh, &fl);
        hdct[(size_t)k * Q4 + d] = T(fh, fl);
      }
    }
  void* d_phit = nullptr;
  e = cudaMalloc(&d_phit, sizeof(T) * J * n3);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error_text("two-fold tables: phit allocation");
    return LBO_ENOMEM;
  }
  if constexpr (sizeof(T) == 16)
    k_widen_f64x2<<<1024, 256>>>(p->d_phit64, (f64x2*)d_phit, (size_t)J * n3);
  else
    k_split_f32x2<<<1024, 256>>>(p->d_phit64, (f32x2*)d_phit, (size_t)J * n3);
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(d_phit);
    return cuda_fail(e, "two-fold tables: phit");
  }
  lbo_status st = upload(hphi, &slot[1]);
  if (st == LBO_OK) st = upload(hom, &slot[2]);
  if (st == LBO_OK) st = upload(hdct, &slot[3]);
  if (st != LBO_OK) {
    cudaFree(d_phit);
    for (int i = 1; i < 4; ++i)
      if (slot[i]) cudaFree(slot[i]), slot[i] = nullptr;
    return st;
  }
  slot[0] = d_phit;
  return LBO_OK;
}

}  // namespace

lbo_status twofold_tables(lbo_plan* p, const void** phi, const void** omega, const void** phit, const void** dct) {
  void** slot = p->precision == LBO_PREC_FP64X2 ? p->d_x2d : p->d_x2f;
  lbo_status st = p->precision == LBO_PREC_FP64X2 ? build<f64x2>(p, slot) : build<f32x2>(p, slot);
  if (st != LBO_OK) return st;
  *phit = slot[0];
  *phi = slot[1];
  *omega = slot[2];
  *dct = slot[3];
  return LBO_OK;
}

void free_twofold_tables(lbo_plan* p) {
  for (int i = 0; i < 4; ++i) {
    if (p->d_x2f[i]) cudaFree(p->d_x2f[i]);
    if (p->d_x2d[i]) cudaFree(p->d_x2d[i]);
    p->d_x2f[i] = p->d_x2d[i] = nullptr;
  }
}

// Built sizes: pairs of FP32 for every N, pairs of FP64 for N = 16 and 32.
static bool twofold_built(int prec, int N) {
  if (prec == LBO_PREC_FP32X2) return N == 16 || N == 24 || N == 32 || N == 48 || N == 64;
  return prec == LBO_PREC_FP64X2 && (N == 16 || N == 32);
}

static lbo_status unsupported(const lbo_plan* p) {
  set_error_text(p->precision == LBO_PREC_FP64X2 ? "FP64X2 is built for N = 16 and 32 only"
                                                 : "two-fold precision: unsupported N");
  return LBO_EUNSUPPORTED;
}

lbo_status run_linearized_twofold(lbo_plan* p, const double* params, const double* g, double* out, int B,
                                  const void* cuh, const void* cw) {
  if (!twofold_built(p->precision, p->N)) return unsupported(p);
  const void* tb[4];
  lbo_status st = twofold_tables(p, &tb[1], &tb[2], &tb[0], &tb[3]);
  if (st != LBO_OK) return st;
  const int b = p->precision == LBO_PREC_FP64X2 ? 2 : 1;
  switch (b * 100 + p->N) {
    case 116: return x2_lin_1_16(p, tb, params, g, out, B, cuh, cw);
    case 124: return x2_lin_1_24(p, tb, params, g, out, B, cuh, cw);
    case 132: return x2_lin_1_32(p, tb, params, g, out, B, cuh, cw);
    case 148: return x2_lin_1_48(p, tb, params, g, out, B, cuh, cw);
    case 164: return x2_lin_1_64(p, tb, params, g, out, B, cuh, cw);
    case 216: return x2_lin_2_16(p, tb, params, g, out, B, cuh, cw);
    case 232: return x2_lin_2_32(p, tb, params, g, out, B, cuh, cw);
    default: return unsupported(p);
  }
}

lbo_status precompute_twofold(lbo_plan* p, const double* params, int B, void* uh, void* w) {
  if (!twofold_built(p->precision, p->N)) return unsupported(p);
  const void* tb[4];
  lbo_status st = twofold_tables(p, &tb[1], &tb[2], &tb[0], &tb[3]);
  if (st != LBO_OK) return st;
  const int b = p->precision == LBO_PREC_FP64X2 ? 2 : 1;
  switch (b * 100 + p->N) {
    case 116: return x2_cache_1_16(p, tb, params, B, uh, w);
    case 124: return x2_cache_1_24(p, tb, params, B, uh, w);
    case 132: return x2_cache_1_32(p, tb, params, B, uh, w);
    case 148: return x2_cache_1_48(p, tb, params, B, uh, w);
    case 164: return x2_cache_1_64(p, tb, params, B, uh, w);
    case 216: return x2_cache_2_16(p, tb, params, B, uh, w);
    case 232: return x2_cache_2_32(p, tb, params, B, uh, w);
    default: return unsupported(p);
  }
}

lbo_status run_quadratic_twofold(lbo_plan* p, QuadState* qs, const double* f, double* out, int B, const void* omg3) {
  if (!twofold_built(p->precision, p->N)) return unsupported(p);
  const void* tb[4];
  lbo_status st = twofold_tables(p, &tb[1], &tb[2], &tb[0], &tb[3]);
  if (st != LBO_OK) return st;
  const int b = p->precision == LBO_PREC_FP64X2 ? 2 : 1;
  switch (b * 100 + p->N) {
    case 116: return x2_quad_1_16(p, qs, tb, f, out, B, omg3);
    case 124: return x2_quad_1_24(p, qs, tb, f, out, B, omg3);
    case 132: return x2_quad_1_32(p, qs, tb, f, out, B, omg3);
    case 148: return x2_quad_1_48(p, qs, tb, f, out, B, omg3);
    case 164: return x2_quad_1_64(p, qs, tb, f, out, B, omg3);
    case 216: return x2_quad_2_16(p, qs, tb, f, out, B, omg3);
    case 232: return x2_quad_2_32(p, qs, tb, f, out, B, omg3);
    default: return unsupported(p);
  }
}

}  // namespace lbo

// build-variants: LBO_X2_B=1:LBO_X2_N=16 LBO_X2_B=1:LBO_X2_N=24 LBO_X2_B=1:LBO_X2_N=32 LBO_X2_B=1:LBO_X2_N=48 LBO_X2_B=1:LBO_X2_N=64 LBO_X2_B=2:LBO_X2_N=16 LBO_X2_B=2:LBO_X2_N=32
//
// L[g] and Q(f,f) on the generic kernels in one two-fold precision and one
// grid size: LBO_X2_B = 1 for pairs of FP32 (FP32X2), 2 for pairs of FP64
// (FP64X2); LBO_X2_N = N.  The build compiles this file once per line entry
// above (each instantiation of the two-fold kernels takes ptxas 10-25 s, so
// one translation unit per size keeps the parallel build short); the pairs
// of FP64 are built for N = 16 and 32, the sizes of the accuracy studies.
// lin_twofold.cu dispatches to the functions defined here.
#include "lin_generic.cuh"
#include "quad_generic.cuh"

#if LBO_X2_B == 1
#define LBO_X2_T f32x2
#else
#define LBO_X2_T f64x2
#endif
#define LBO_CAT4_(a, b, c, d) a##b##c##d
#define LBO_CAT4(a, b, c, d) LBO_CAT4_(a, b, c, d)

namespace lbo {

lbo_status LBO_CAT4(x2_lin_, LBO_X2_B, _, LBO_X2_N)(lbo_plan* p, const void* const* tb, const double* params,
                                                    const double* g, double* out, int B, const void* cuh,
                                                    const void* cw) {
  cudaError_t e = upload_twiddles();  // this translation unit's copy
  if (e != cudaSuccess) return cuda_fail(e, "two-fold twiddles");
  using T = LBO_X2_T;
  GenericTables<T> t{(const T*)tb[1], (const T*)tb[2], (const T*)tb[0], (const T*)tb[3]};
  GenericCache<T> mc{(const T*)cuh, (const T*)cw};
  return run_linearized_generic<T, LBO_X2_N>(p, t, params, g, out, B, p->ws, cuh ? &mc : nullptr);
}

lbo_status LBO_CAT4(x2_cache_, LBO_X2_B, _, LBO_X2_N)(lbo_plan* p, const void* const* tb, const double* params,
                                                      int B, void* uh, void* w) {
  cudaError_t e = upload_twiddles();
  if (e != cudaSuccess) return cuda_fail(e, "two-fold twiddles");
  using T = LBO_X2_T;
  GenericTables<T> t{(const T*)tb[1], (const T*)tb[2], (const T*)tb[0], (const T*)tb[3]};
  return precompute_maxwellian_generic<T, LBO_X2_N>(p, t, params, B, p->ws, (T*)uh, (T*)w);
}

lbo_status LBO_CAT4(x2_quad_, LBO_X2_B, _, LBO_X2_N)(lbo_plan* p, QuadState* qs, const void* const* tb,
                                                     const double* f, double* out, int B, const void* omg3) {
  cudaError_t e = upload_twiddles();
  if (e != cudaSuccess) return cuda_fail(e, "two-fold twiddles");
  using T = LBO_X2_T;
  return run_quadratic<T, LBO_X2_N>(p, qs, f, out, B, (const T*)tb[1], (const T*)tb[2], (const T*)omg3);
}

}  // namespace lbo

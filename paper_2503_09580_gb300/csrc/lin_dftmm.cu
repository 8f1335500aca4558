// L[g] with every transform of Algorithm 1 as a dense DFT contraction on the
// tensor cores (dftmm.cuh): precisions LBO_PREC_BF16_SPLIT and
// LBO_PREC_FP16_SPLIT, N = 16, 32, 64.
//
// Fields are full complex FP32 arrays [B][N^3] (a real field is stored with
// zero imaginary parts), transformed in place one axis per launch; the
// pointwise stages of Algorithm 1 ride on the passes:
//   r^    = F1 F2 F3 (r),  r = g/M with the cut-off formed in the first pass
//   per radial node j:
//     psi_j = Re F3^-1 F2^-1 F1^-1 (u^_j r^ / N^3)
//     L^+  += phi_j F1 F2 F3 (M^h psi_j)        (phi_j carries 1/N^3)
//   L+ = Re F3^-1 F2^-1 F1^-1 (L^+),  u = Re F^-1 (omega F(g))
//   out = L+ - u M - w g  (FP64)
// u^_j and w = InvFFT(omega FFT(M)) come from the Maxwellian cache
// (lbo_plan_cache_maxwellians) when it holds this call's Maxwellians, else
// they are computed by the generic FP32 kernels for this call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dftmm.cuh"
#include "lin_generic.cuh"

namespace lbo {
namespace {

using mm::PassArgs;

// Shared-memory image of W_hi then W_lo (umma.cuh layout) for a length-N
// DFT as a real (2N x 2N) matrix: forward exp(-2 pi i q (j - N/2) / N) from a
// centred real-space axis to a cyclic frequency axis, inverse the conjugate
// (frequency -> real space).  Entries from the double-pair twiddle table.
std::vector<uint16_t> w_image(int N, bool inverse, bool bf) {
  const int K = 2 * N;
  std::vector<uint16_t> img((size_t)2 * K * K);
  uint16_t* hi = img.data();
  uint16_t* lo = img.data() + (size_t)K * K;
  auto put = [&](int o, int k, double v) {
    const float f = (float)v;
    uint16_t h, l;
    if (bf) {
      const __nv_bfloat16 bh = __float2bfloat16_rn(f);
      h = __bfloat16_as_ushort(bh);
      l = __bfloat16_as_ushort(__float2bfloat16_rn((float)(v - (double)__bfloat162float(bh))));
    } else {
      const __half hh = __float2half_rn(f);
      h = __half_as_ushort(hh);
      l = __half_as_ushort(__float2half_rn((float)(v - (double)__half2float(hh))));
    }
    const uint32_t off = umma::kmajor_offset(o, k, K) / 2;
    hi[off] = h;
    lo[off] = l;
  };
  for (int q = 0; q < N; ++q)
    for (int j = 0; j < N; ++j) {
      // exp(-2 pi i q j / N) from the table, times (-1)^q for the centred index
      const int m = (int)(((64 / N) * (long)q * j) % 64);
      double a = kTw64Hi[m][0], b = kTw64Hi[m][2];
      if (q & 1) a = -a, b = -b;
      if (inverse) b = -b;
      // forward: row q (output), column j (input); inverse: row j, column q
      const int o = inverse ? j : q, k = inverse ? q : j;
      put(2 * o, 2 * k, a);
      put(2 * o, 2 * k + 1, -b);
      put(2 * o + 1, 2 * k, b);
      put(2 * o + 1, 2 * k + 1, a);
    }
  return img;
}

template <int N, int AXIS, int PRE, int POST, bool BF>
lbo_status pass(lbo_plan* p, const char* name, PassArgs a, int sms) {
  using G = mm::Geo<N>;
  auto k = mm::k_dft_pass<N, AXIS, PRE, POST, BF>;
  raise_smem_limit((const void*)k, G::SMEM);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, mm::kTile, G::SMEM);
  per_sm = std::max(1, std::min(per_sm, 512 / G::TMEM_COLS));  // TMEM columns of the SM
  const size_t tiles = (size_t)a.B * N * N / mm::kTile;
  const int grid = (int)std::min<size_t>(tiles, (size_t)sms * per_sm);
  LBO_LAUNCH(p, name, p->stream, k, grid, mm::kTile, G::SMEM, a);
  return LBO_OK;
}

// out = L+ - u M - w g (FP64): L+, u FP64 fields, w FP32; grid (N, B)
template <int N>
__global__ void __launch_bounds__(256) k_tc_combine(const double* __restrict__ params, const double* __restrict__ g,
                                                    const double* __restrict__ Lp, const double* __restrict__ uu,
                                                    const float* __restrict__ ww, double* __restrict__ out, double h,
                                                    double log_inv_eps) {
  __shared__ double em[3 * N];
  __shared__ double thr;
  const int b = blockIdx.y, i1 = blockIdx.x;
  const InstanceParams q = load_params(params, b);
  fill_maxwellian_tables<N>(em, &thr, q, h, log_inv_eps);
  const size_t base = ((size_t)b * N + i1) * N * N;
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    const double M = em[i1] * em[N + t / N] * em[2 * N + t % N];
    const size_t o = base + t;
    out[o] = Lp[o] - uu[o] * M - (double)ww[o] * g[o];
  }
}

template <int N, bool BF>
lbo_status run(lbo_plan* p, const double* params, const double* g, double* out, int B, const float* uh,
               const float* w, unsigned char* ws, const uint16_t* wf, const uint16_t* wi, int* err) {
  using namespace mm;
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t n3 = (size_t)N * N * N, HC3 = (size_t)(N / 2 + 1) * (N / 2 + 1) * (N / 2 + 1);
  float2* RH = (float2*)ws;
  float2* W1 = RH + (size_t)B * n3;
  float2* LH = W1 + (size_t)B * n3;
  double* R1 = (double*)(LH + (size_t)B * n3);
  double* R2 = R1 + (size_t)B * n3;
  const int Q = 3 * (N / 2) * (N / 2) + 1;
  PassArgs a{};
  a.params = params;
  a.g = g;
  a.err = err;
  a.h = 2.0 * p->L / N;
  a.log_inv_eps = std::log(1.0 / p->eps);
  a.cutoff = p->cutoff;
  a.B = B;
  auto fwd = [&](PassArgs x) { x.wmat = wf; return x; };
  auto inv = [&](PassArgs x) { x.wmat = wi; return x; };
  PassArgs t;
  // r^ = F(r), r formed from g in the first pass
  t = fwd(a), t.dst = RH;
  pass<N, 3, PRE_RATIO, POST_STORE, BF>(p, "tc_fwd3_ratio", t, sms);
  t = fwd(a), t.src = RH, t.dst = RH;
  pass<N, 2, PRE_NONE, POST_STORE, BF>(p, "tc_fwd2", t, sms);
  pass<N, 1, PRE_NONE, POST_STORE, BF>(p, "tc_fwd1", t, sms);
  int launches = 3;
  for (int j = 0; j < p->J; ++j) {
    t = inv(a), t.src = RH, t.dst = W1, t.uhat = uh + (size_t)j * B * HC3, t.scale = 1.0f / (float)n3;
    pass<N, 1, PRE_UHAT, POST_STORE, BF>(p, "tc_inv1_uhat", t, sms);
    t = inv(a), t.src = W1, t.dst = W1;
    pass<N, 2, PRE_NONE, POST_STORE, BF>(p, "tc_inv2", t, sms);
    pass<N, 3, PRE_NONE, POST_REAL, BF>(p, "tc_inv3_real", t, sms);
    t = fwd(a), t.src = W1, t.dst = W1;
    pass<N, 3, PRE_MH, POST_STORE, BF>(p, "tc_fwd3_mh", t, sms);
    pass<N, 2, PRE_NONE, POST_STORE, BF>(p, "tc_fwd2", t, sms);
    t = fwd(a), t.src = W1, t.dst = LH, t.table = p->d_phi32 + (size_t)j * Q, t.first = j == 0;
    pass<N, 1, PRE_NONE, POST_ACC, BF>(p, "tc_fwd1_acc", t, sms);
    launches += 6;
  }
  // L+ = F^-1 (L^+)
  t = inv(a), t.src = LH, t.dst = LH;
  pass<N, 1, PRE_NONE, POST_STORE, BF>(p, "tc_inv1", t, sms);
  pass<N, 2, PRE_NONE, POST_STORE, BF>(p, "tc_inv2", t, sms);
  t.dst64 = R1;
  pass<N, 3, PRE_NONE, POST_REAL64, BF>(p, "tc_inv3_real64", t, sms);
  // loss: u = F^-1 (omega F(g))
  t = fwd(a), t.dst = W1;
  pass<N, 3, PRE_REAL64, POST_STORE, BF>(p, "tc_fwd3_g", t, sms);
  t = fwd(a), t.src = W1, t.dst = W1;
  pass<N, 2, PRE_NONE, POST_STORE, BF>(p, "tc_fwd2", t, sms);
  t.table = p->d_omega32;
  pass<N, 1, PRE_NONE, POST_TABLE, BF>(p, "tc_fwd1_omega", t, sms);
  t = inv(a), t.src = W1, t.dst = W1;
  pass<N, 1, PRE_NONE, POST_STORE, BF>(p, "tc_inv1", t, sms);
  pass<N, 2, PRE_NONE, POST_STORE, BF>(p, "tc_inv2", t, sms);
  t.dst64 = R2;
  pass<N, 3, PRE_NONE, POST_REAL64, BF>(p, "tc_inv3_real64", t, sms);
  LBO_LAUNCH(p, "tc_combine", p->stream, k_tc_combine<N>, dim3(N, B), 256, 0, params, g, R1, R2, w, out, a.h,
             a.log_inv_eps);
  launches += 13;
  p->last_launches += launches;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "tensor-core linearized launch");
}

}  // namespace

// bytes of the pass workspace: three complex FP32 fields and two FP64 fields
size_t dftmm_workspace_bytes(int N, int B) {
  const size_t n3 = (size_t)N * N * N;
  return (size_t)B * n3 * (3 * 8 + 2 * 8);
}

// W images of the plan (forward, inverse) for its precision, built once
static lbo_status w_images(lbo_plan* p, const uint16_t** wf, const uint16_t** wi) {
  const bool bf = p->precision == LBO_PREC_BF16_SPLIT;
  void** slot = bf ? p->d_wbf : p->d_wfp;
  if (!slot[0]) {
    for (int d = 0; d < 2; ++d) {
      std::vector<uint16_t> img = w_image(p->N, d == 1, bf);
      cudaError_t e = cudaMalloc(&slot[d], img.size() * sizeof(uint16_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(slot[d], img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        for (int i = 0; i < 2; ++i)
          if (slot[i]) cudaFree(slot[i]), slot[i] = nullptr;
        return cuda_fail(e, "tensor-core DFT matrices");
      }
    }
  }
  *wf = (const uint16_t*)slot[0];
  *wi = (const uint16_t*)slot[1];
  return LBO_OK;
}

void free_dftmm(lbo_plan* p) {
  for (int i = 0; i < 2; ++i) {
    if (p->d_wbf[i]) cudaFree(p->d_wbf[i]);
    if (p->d_wfp[i]) cudaFree(p->d_wfp[i]);
    p->d_wbf[i] = p->d_wfp[i] = nullptr;
  }
  if (p->d_tc_err) cudaFree(p->d_tc_err);
  p->d_tc_err = nullptr;
}

bool dftmm_supported(int N) { return N == 16 || N == 32 || N == 64; }

lbo_status run_linearized_dftmm(lbo_plan* p, const double* params, const double* g, double* out, int B,
                                const float* uh, const float* w, void* ws) {
  if (!dftmm_supported(p->N)) {
    set_error_text("split 16-bit tensor-core precisions: N = 16, 32 or 64");
    return LBO_EUNSUPPORTED;
  }
  const uint16_t *wf, *wi;
  lbo_status st = w_images(p, &wf, &wi);
  if (st != LBO_OK) return st;
  if (!p->d_tc_err) {
    cudaError_t e = cudaMalloc(&p->d_tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_tc_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core error flag");
  }
  int* err = (int*)p->d_tc_err;
  unsigned char* wsb = (unsigned char*)ws;
  const bool bf = p->precision == LBO_PREC_BF16_SPLIT;
  switch (p->N * 2 + (bf ? 1 : 0)) {
    case 33: return run<16, true>(p, params, g, out, B, uh, w, wsb, wf, wi, err);
    case 32: return run<16, false>(p, params, g, out, B, uh, w, wsb, wf, wi, err);
    case 65: return run<32, true>(p, params, g, out, B, uh, w, wsb, wf, wi, err);
    case 64: return run<32, false>(p, params, g, out, B, uh, w, wsb, wf, wi, err);
    case 129: return run<64, true>(p, params, g, out, B, uh, w, wsb, wf, wi, err);
    case 128: return run<64, false>(p, params, g, out, B, uh, w, wsb, wf, wi, err);
    default: return LBO_EUNSUPPORTED;
  }
}

// Did a tensor-core pass give up waiting for an MMA since the last check?
// (Synchronizes the plan's stream; clears the flag.)
lbo_status dftmm_check(lbo_plan* p) {
  if (!p->d_tc_err) return LBO_OK;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, p->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core error flag");
  if (h) {
    cudaMemsetAsync(p->d_tc_err, 0, sizeof(int), p->stream);
    set_error_text("tensor-core pass: an MMA did not complete within the wait limit");
    return LBO_ETIMEOUT;
  }
  return LBO_OK;
}

}  // namespace lbo

using namespace lbo;

namespace {
template <int N, int AXIS, bool BF>
lbo_status one_pass(lbo_plan* p, const float* in, float* out, int batch, const uint16_t* wm, int* err, int sms) {
  PassArgs a{};
  a.src = (const float2*)in;
  a.dst = (float2*)out;
  a.wmat = wm;
  a.err = err;
  a.B = batch;
  return pass<N, AXIS, mm::PRE_NONE, mm::POST_STORE, BF>(p, "tc_axis", a, sms);
}
}  // namespace

extern "C" lbo_status lbo_dft_axis_tensor(int N, int precision, int inverse, int axis, const float* in, float* out,
                                          int batch, void* stream) {
  if (!dftmm_supported(N) || (precision != LBO_PREC_BF16_SPLIT && precision != LBO_PREC_FP16_SPLIT))
    return LBO_EUNSUPPORTED;
  if (!in || !out || batch < 0 || axis < 1 || axis > 3) return LBO_EINVAL;
  if (batch == 0) return LBO_OK;
  lbo_plan tmp;  // carries the stream, the precision and the matrices for this call only
  tmp.N = N;
  tmp.precision = precision;
  tmp.stream = (cudaStream_t)stream;
  const uint16_t *wf, *wi;
  lbo_status st = w_images(&tmp, &wf, &wi);
  int* err = nullptr;
  if (st == LBO_OK && cudaMalloc(&err, sizeof(int)) != cudaSuccess) st = LBO_ENOMEM;
  if (st == LBO_OK) cudaMemset(err, 0, sizeof(int));
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint16_t* wm = inverse ? wi : wf;
  const bool bf = precision == LBO_PREC_BF16_SPLIT;
  if (st == LBO_OK) {
    const int key = N * 100 + axis * 10 + (bf ? 1 : 0);
    switch (key) {
#define LBO_ONE(n, ax)                                                                     \
  case n * 100 + ax * 10 + 1: st = one_pass<n, ax, true>(&tmp, in, out, batch, wm, err, sms); break; \
  case n * 100 + ax * 10 + 0: st = one_pass<n, ax, false>(&tmp, in, out, batch, wm, err, sms); break;
      LBO_ONE(16, 1) LBO_ONE(16, 2) LBO_ONE(16, 3)
      LBO_ONE(32, 1) LBO_ONE(32, 2) LBO_ONE(32, 3)
      LBO_ONE(64, 1) LBO_ONE(64, 2) LBO_ONE(64, 3)
#undef LBO_ONE
      default: st = LBO_EUNSUPPORTED;
    }
  }
  cudaError_t e = cudaStreamSynchronize(tmp.stream);
  if (st == LBO_OK && e != cudaSuccess) st = cuda_fail(e, "tensor-core axis pass");
  if (st == LBO_OK && err) {
    int h = 0;
    cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (h) {
      set_error_text("tensor-core pass: an MMA did not complete within the wait limit");
      st = LBO_ETIMEOUT;
    }
  }
  if (err) cudaFree(err);
  free_dftmm(&tmp);
  return st;
}

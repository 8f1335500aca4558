// lbo_apply_linearized_noalloc: the linearized operator of
// lbo_apply_linearized with its scratch buffers taken from a fixed
// file-scope device array instead of memory the plan allocates.
//
// Who needs it: callers that must not allocate device memory when they
// apply the operator -- code that runs between the set-up and tear-down of
// a fixed memory budget (e.g. a solver whose pools are sized at start-up
// and may not grow), real-time or embedded loops where cudaMalloc's
// implicit device synchronisation and unbounded latency are not allowed,
// and hosts that forbid allocation after initialisation.  The regular
// entry point grows its workspace with cudaMalloc whenever a batch is
// larger than any seen before; this one never allocates.
//
// Limits and behaviour:
//  * The scratch is one static __device__ array of LBO_NOALLOC_SCRATCH_BYTES
//    (64 MiB) in this library; every GPU that loads the library holds it
//    until the process exits.  A call whose batch needs more (batch *
//    lbo_noalloc_bytes_per_instance) is rejected with LBO_EINVAL before
//    any launch.
//  * Every call shares the array and it keeps the last call's contents.
//    No part of it has to start at zero: every buffer is written in full
//    before it is read within one call.  Calls that overlap on the GPU
//    (e.g. on two streams at once) race on the array and give wrong
//    results; serialise them.
//  * The first call on a device, with that device current, looks up the
//    array's device address (cudaGetSymbolAddress) and uploads this file's
//    FFT twiddle table; make that first call before any stream capture.
//  * It always runs the generic plane/axis kernel set (the one
//    LBO_OPT_KERNEL = 1 selects), also where the regular entry point would
//    pick the fused FP32 kernels (N = 32), and only the FP64 and FP32
//    precisions.
//  * The device current at the call must be the plan's device (the plan's
//    tables live there); other devices are rejected.
//  * Arrays must be device pointers; the plan's tables must be current
//    (a plan whose R, C or hemisphere option changed since its last
//    lbo_apply_linearized call is rejected, since rebuilding the tables
//    allocates).  Nothing here calls cudaMalloc, cudaFree or an allocating
//    library routine.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "lbo_internal.h"
#include "lin_kernels.cuh"

#define LBO_NOALLOC_SCRATCH_BYTES (64ull << 20)

namespace lbo {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LBO_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device
bool g_ready[kMaxDevices] = {};
std::mutex g_setup_mutex;  // two host threads making their first call at once

// Per-device set-up: the array's address and this file's twiddle table.
lbo_status setup_device(int dev) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error_text("noalloc: device index out of range");
    return LBO_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_ready[dev]) return LBO_OK;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || ptr == nullptr) return cuda_fail(e, "noalloc: cudaGetSymbolAddress");
  e = upload_twiddles_now();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc: twiddle upload");
  g_scratch_ptr[dev] = ptr;
  g_ready[dev] = true;
  return LBO_OK;
}

size_t bytes_per_instance(int N, bool f64) {
  const size_t H = (size_t)N * N * (N / 2 + 1), n3 = (size_t)N * N * N, HN = N / 2 + 1;
  const size_t re = f64 ? 8 : 4;
  return 3 * H * 2 * re + 3 * n3 * re + HN * HN * HN * re;
}

bool on_device(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <int N>
struct PPC_ { static constexpr int v = N == 16 ? 8 : (N == 32 ? 4 : (N == 24 ? 4 : (N == 48 ? 2 : 1))); };

template <typename K>
void smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Same launch sequence as the regular entry point, scratch from `ws`.
template <typename T, int N>
lbo_status run(const lbo_plan* p, const double* params, const double* g, double* out, int B, unsigned char* ws) {
  constexpr int PPC = PPC_<N>::v, CW = 32, HC = N / 2 + 1;
  const size_t H = (size_t)N * N * HC, n3 = (size_t)N * N * N;
  const int Q = 3 * (N / 2) * (N / 2) + 1;
  cudaStream_t s = p->stream;
  cpx<T>* RH = (cpx<T>*)ws;
  cpx<T>* W1 = RH + (size_t)B * H;
  cpx<T>* LH = W1 + (size_t)B * H;
  T* R1 = (T*)(LH + (size_t)B * H);
  T* R2 = R1 + (size_t)B * n3;
  T* R3 = R2 + (size_t)B * n3;
  T* UP = R3 + (size_t)B * n3;
  const bool f64 = sizeof(T) == 8;
  const T* dct = (const T*)(f64 ? (const void*)p->d_dct64 : (const void*)p->d_dct32);
  const T* phi = (const T*)(f64 ? (const void*)p->d_phi64 : (const void*)p->d_phi32);
  const T* omg = (const T*)(f64 ? (const void*)p->d_omega64 : (const void*)p->d_omega32);
  const T* phit = (const T*)(f64 ? (const void*)p->d_phit64 : (const void*)p->d_phit32);
  const size_t sm = PlaneSmem<T, N, PPC>::BYTES;
  const dim3 gp(N / PPC, B), ga((N * HC + CW - 1) / CW, B), blk(256);
  auto kf_ratio = k_plane_fwd<T, N, PPC, SRC_RATIO>;
  constexpr int PL = UhatPlanes<N>::PL;
  auto k_up = k_uhat_planes<T, N, PL>;
  const size_t sm_up = sizeof(T) * ((size_t)PL * HC * HC + (size_t)HC * (N / 4));
  auto kf_real = k_plane_fwd<T, N, PPC, SRC_REAL64>;
  auto kf_maxw = k_plane_fwd<T, N, PPC, SRC_MAXW>;
  auto ki_mh = k_plane_inv<T, N, PPC, INV_MH_FWD>;
  auto ki_real = k_plane_inv<T, N, PPC, INV_TO_REAL>;
  smem_attr(kf_ratio, sm);
  smem_attr(k_up, sm_up);
  smem_attr(kf_real, sm);
  smem_attr(kf_maxw, sm);
  smem_attr(ki_mh, sm);
  smem_attr(ki_real, sm);
  PlaneArgs pa{};
  pa.params = params;
  pa.g = g;
  pa.h = 2.0 * p->L / N;
  pa.log_inv_eps = std::log(1.0 / p->eps);
  pa.cutoff = p->cutoff;
  Axis1Args ax{};
  kf_ratio<<<gp, blk, sm, s>>>(pa, W1);
  k_axis1<T, N, CW, AX_FWD_STORE><<<ga, blk, 0, s>>>(ax, W1, RH);
  for (int j = 0; j < p->J; ++j) {
    k_up<<<dim3((HC + PL - 1) / PL, B), blk, sm_up, s>>>(params, phit + (size_t)j * n3, dct, pa.h, UP);
    Axis1Args a1{};
    a1.uplanes = UP;
    a1.dct = dct;
    a1.scale = 1.0 / (double)n3;
    k_axis1<T, N, CW, AX_UHAT_INV><<<ga, blk, 0, s>>>(a1, RH, W1);
    ki_mh<<<gp, blk, sm, s>>>(pa, W1, (T*)nullptr);
    Axis1Args a2{};
    a2.table = phi + (size_t)j * Q;
    a2.first = j == 0;
    k_axis1<T, N, CW, AX_FWD_ACC><<<ga, blk, 0, s>>>(a2, W1, LH);
  }
  k_axis1<T, N, CW, AX_INV_STORE><<<ga, blk, 0, s>>>(ax, LH, LH);
  ki_real<<<gp, blk, sm, s>>>(pa, LH, R1);
  Axis1Args a3{};
  a3.table = omg;
  kf_real<<<gp, blk, sm, s>>>(pa, W1);
  k_axis1<T, N, CW, AX_FWD_MULT_INV><<<ga, blk, 0, s>>>(a3, W1, W1);
  ki_real<<<gp, blk, sm, s>>>(pa, W1, R2);
  kf_maxw<<<gp, blk, sm, s>>>(pa, W1);
  k_axis1<T, N, CW, AX_FWD_MULT_INV><<<ga, blk, 0, s>>>(a3, W1, W1);
  ki_real<<<gp, blk, sm, s>>>(pa, W1, R3);
  k_combine<T, N><<<dim3(N, B), 256, 0, s>>>(params, g, R1, R2, R3, out, pa.h, pa.log_inv_eps);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "noalloc launch");
}

template <typename T>
lbo_status dispatch(const lbo_plan* p, const double* params, const double* g, double* out, int B,
                    unsigned char* ws) {
  switch (p->N) {
    case 16: return run<T, 16>(p, params, g, out, B, ws);
    case 24: return run<T, 24>(p, params, g, out, B, ws);
    case 32: return run<T, 32>(p, params, g, out, B, ws);
    case 48: return run<T, 48>(p, params, g, out, B, ws);
    case 64: return run<T, 64>(p, params, g, out, B, ws);
    default: return LBO_EUNSUPPORTED;
  }
}

}  // namespace
}  // namespace lbo

extern "C" {

size_t lbo_noalloc_scratch_bytes(void) { return (size_t)LBO_NOALLOC_SCRATCH_BYTES; }

size_t lbo_noalloc_bytes_per_instance(const lbo_plan* p) {
  if (!p) return 0;
  return lbo::bytes_per_instance(p->N, p->precision == LBO_PREC_FP64);
}

lbo_status lbo_apply_linearized_noalloc(lbo_plan* p, const double* params, const double* g, double* out,
                                        int batch) {
  if (!p || batch < 0) return LBO_EINVAL;
  if (batch == 0) {
    p->last_launches = 0;
    return LBO_OK;
  }
  if (!params || !g || !out || out == g) return LBO_EINVAL;
  if (p->mass_fix || p->moment_fix) {
    lbo::set_error_text("noalloc: mass/moment fix options are not supported by this entry point");
    return LBO_EUNSUPPORTED;
  }
  if (p->precision != LBO_PREC_FP64 && p->precision != LBO_PREC_FP32) {
    lbo::set_error_text("noalloc: only the FP64 and FP32 precisions are supported by this entry point");
    return LBO_EUNSUPPORTED;
  }
  if (p->tables_dirty) {
    lbo::set_error_text("noalloc: plan tables are out of date (rebuilding them allocates)");
    return LBO_EINVAL;
  }
  const size_t need = (size_t)batch * lbo_noalloc_bytes_per_instance(p);
  if (need > (size_t)LBO_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof(msg), "noalloc: batch %d needs %zu bytes of scratch, above the %llu-byte static scratch",
             batch, need, (unsigned long long)LBO_NOALLOC_SCRATCH_BYTES);
    lbo::set_error_text(msg);
    return LBO_EINVAL;
  }
  if (!lbo::on_device(params) || !lbo::on_device(g) || !lbo::on_device(out)) {
    lbo::set_error_text("noalloc: arrays must be device pointers");
    return LBO_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbo::cuda_fail(e, "noalloc: cudaGetDevice");
  if (dev != p->device) {
    lbo::set_error_text("noalloc: the current device is not the plan's device");
    return LBO_EINVAL;
  }
  lbo_status st = lbo::setup_device(dev);
  if (st != LBO_OK) return st;
  unsigned char* ws = (unsigned char*)lbo::g_scratch_ptr[dev];
  st = p->precision == LBO_PREC_FP64 ? lbo::dispatch<double>(p, params, g, out, batch, ws)
                                     : lbo::dispatch<float>(p, params, g, out, batch, ws);
  // same count as the regular generic path: 2 + 4 per radial node + 9
  p->last_launches = st == LBO_OK ? 4 * p->J + 11 : 0;
  return st;
}

}  // extern "C"

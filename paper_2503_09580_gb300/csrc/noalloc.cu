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
//    LBO_OPT_KERNEL = 1 selects; the same launch sequence, lin_generic.cuh),
//    also where the regular entry point would pick the fused FP32 kernels
//    (N = 32), and only the FP64 and FP32 precisions.
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
#include "lin_generic.cuh"

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
  void* ws = lbo::g_scratch_ptr[dev];
  // the launch sequence of the regular generic path, scratch from the array;
  // per-kernel profiling is held off (its events would be created here)
  const bool prof = p->profiling;
  p->profiling = false;
  st = p->precision == LBO_PREC_FP64
           ? lbo::dispatch_generic<double>(p, lbo::plain_tables<double>(p), params, g, out, batch, ws)
           : lbo::dispatch_generic<float>(p, lbo::plain_tables<float>(p), params, g, out, batch, ws);
  p->profiling = prof;
  if (st != LBO_OK) p->last_launches = 0;
  return st;
}

}  // extern "C"

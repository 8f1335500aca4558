// lbo_measure_alu_peaks: dense FP32 FFMA and FP64 DFMA throughput of the
// current device, measured with CUDA events (the denominators of the
// library's roofline fractions for the ALU-bound kernels).
//
// Every thread runs ACC independent fused multiply-add chains
// x <- x * a + b (a = 1 - 2^-10, b = 2^-10: normal numbers throughout, no
// overflow), enough independent work to hide the pipe latency; the grid is
// SMs x 8 blocks of 256 threads (one full wave, 64 warps per SM).  The rate
// such a loop reaches depends on its code shape, not on the operand values:
// - the FP32 pipe is issue-bound, so loop overhead in the same issue slots
//   costs rate (6 % with 4-fold unrolling): the loop is unrolled 16 times;
// - on GB300 a DFMA whose operands are all registers issues about 19 %
//   faster than one that reads a constant-bank operand (a compile-time
//   constant, or a kernel parameter at some offsets: the same loop measured
//   1.20 or 1.01 TFLOP/s depending only on the kernel's parameter list).  So
//   a and b are read from a constant table through an index the compiler
//   cannot see (blockDim.x >> 12, always 0), which puts them in registers.
// A store that depends on every chain keeps the work alive.  In the FP32
// run thread 0 of every block reads clock64() around its loop; the longest
// loop over the blocks of the single wave, divided by the event time, gives
// the SM clock the peaks were measured at.
#include <cuda_runtime.h>

#include <algorithm>

#include "lbo_internal.h"

namespace lbo {
namespace {

constexpr int kThreads = 256, kBlocksPerSM = 8;

static __constant__ double c_ab64[2] = {1.0 - 1.0 / 1024.0, 1.0 / 1024.0};
static __constant__ float c_ab32[2] = {1.0f - 1.0f / 1024.0f, 1.0f / 1024.0f};

// CLK: thread 0 of every block brackets its loop with clock64().
template <typename T, int ACC, bool CLK>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* sink, long long* cycles, int iters) {
  const int z = (int)(blockDim.x >> 12);
  const T* ab = sizeof(T) == 8 ? (const T*)c_ab64 : (const T*)c_ab32;
  const T a = ab[z], b = ab[z + 1];
  T x[ACC];
#pragma unroll
  for (int i = 0; i < ACC; ++i) x[i] = (T)(threadIdx.x + 1) * (T)(i + 1) * (T)0.0009765625;
  long long c0 = 0;
  if constexpr (CLK) c0 = clock64();
#pragma unroll 16
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < ACC; ++i) x[i] = fma(x[i], a, b);
  }
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < ACC; ++i) s += x[i];
  if (s == (T)-1) sink[blockIdx.x * kThreads + threadIdx.x] = s;  // never taken: x stays near 1
  if constexpr (CLK) {
    const long long c1 = clock64();
    if (threadIdx.x == 0) atomicMax((unsigned long long*)cycles, (unsigned long long)(c1 - c0));
  }
}

// Best rate (TFLOP/s) of k_fma_chains<T, ACC, CLK> over three launches; with
// CLK, *mhz is the clock of the best.
template <typename T, int ACC, bool CLK>
lbo_status measure(cudaStream_t s, int sms, int iters, double* best, double* mhz, T* sink, long long* d_cyc) {
  const int blocks = sms * kBlocksPerSM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "peaks: event");
  }
  k_fma_chains<T, ACC, CLK><<<blocks, kThreads, 0, s>>>(sink, d_cyc, iters / 8);  // warm-up
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaMemsetAsync(d_cyc, 0, sizeof(long long), s);
    cudaEventRecord(e0, s);
    k_fma_chains<T, ACC, CLK><<<blocks, kThreads, 0, s>>>(sink, d_cyc, iters);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long cyc = 0;
    e = cudaMemcpy(&cyc, d_cyc, sizeof(cyc), cudaMemcpyDeviceToHost);
    const double flops = 2.0 * ACC * (double)iters * blocks * kThreads;
    const double rate = flops / (ms * 1e-3) / 1e12;
    if (rate > *best) {
      *best = rate;
      if (CLK) *mhz = (double)cyc / (ms * 1e-3) / 1e6;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "peaks: kernel");
}

}  // namespace
}  // namespace lbo

extern "C" lbo_status lbo_measure_alu_peaks(void* stream, double* fp32_tflops, double* fp64_tflops, int* sm_count,
                                            double* sm_mhz) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return lbo::cuda_fail(e, "peaks: device");
  cudaStream_t s = (cudaStream_t)stream;
  double* sink = nullptr;
  long long* cyc = nullptr;
  const size_t n = (size_t)sms * lbo::kBlocksPerSM * lbo::kThreads;
  e = cudaMalloc(&sink, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&cyc, sizeof(long long));
  if (e != cudaSuccess) {
    if (sink) cudaFree(sink);
    cudaGetLastError();
    return LBO_ENOMEM;
  }
  // about 25 ms per launch on a GB300 (128 FP32 and about 2 FP64 FMA lanes per SM)
  double f32 = 0, f64 = 0, mhz32 = 0, mhz64 = 0;
  lbo_status st = lbo::measure<float, 8, true>(s, sms, 1 << 19, &f32, &mhz32, (float*)sink, cyc);
  if (st == LBO_OK) st = lbo::measure<double, 8, false>(s, sms, 1 << 13, &f64, &mhz64, sink, cyc);
  cudaFree(sink);
  cudaFree(cyc);
  if (st != LBO_OK) return st;
  if (fp32_tflops) *fp32_tflops = f32;
  if (fp64_tflops) *fp64_tflops = f64;
  if (sm_count) *sm_count = sms;
  if (sm_mhz) *sm_mhz = std::max(mhz32, mhz64);
  return LBO_OK;
}

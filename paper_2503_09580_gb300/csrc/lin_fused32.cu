// Fused FP32 path of Algorithm 1 for N = 32.
//
// One CTA holds the half spectrum of one instance (32 x 32 x 17 complex
// FP32 = 139 KB of shared memory) and runs the gain-term loop for a group
// of radial nodes j entirely on chip.  Every axis pass is one in-register
// 32-point FFT per thread (544 threads = one pencil each):
//   rows   (i1, q):  two real rows 2q, 2q+1 packed as one complex row,
//                    transformed along i3 and split into two half rows;
//   axis 2 (i1, k3): pencil along i2;   axis 1 (i2, k3): pencil along i1.
// The shared-memory layout is the one of fused32.cuh.  Spectra are in
// natural frequency order (the register FFT has no permutation cost), so r^
// and the partial sums use the same index.
//
// Kernels per application of a batch: k_f32_head (r^ = FFT(r) / N^3),
// k_f32_uhat (u^_j = FFT(M^g phit_j) of every instance and radial node, as
// a DCT-I of one octant), k_f32_gain (grid = (j-groups + 1) x batch: partial
// L^+ per group, and the loss term written to an FP32 buffer by the extra
// block), k_f32_tail (sum of the partials, inverse transform, plus the loss
// term, written to out in FP64).
#include <cmath>

#include "fused32.cuh"
#include "lbo_internal.h"
#include "tmem.cuh"
#include "umma.cuh"

namespace lbo {
namespace {
using namespace f32;

struct FusedArgs {
  const double* params;
  const double* g;
  const float* phit;   // [J][N^3] cyclic displacement order
  const float* phi;    // [J][QMAX], pre-scaled by N^-3
  const float* omega;  // [QMAX], pre-scaled by N^-3
  cpx<float>* rhat;    // [B][F_H], pre-scaled by N^-3
  cpx<float>* part;    // [G][B][F_H] partial L^+ per j-group
  float* uhat;         // [B][J][U_STRIDE] u^_j = FFT(M^g phit_j) on the octant k in [0,16]^3
  float* lossf;        // [B][N^3] loss term -u M - w g in FP32 (loss block -> tail)
  double* out;         // [B][N^3]
  int* err;            // set when a bounded wait gave up (read by lbo_plan_sync)
  double h, log_inv_eps;
  int cutoff, J, G, B, Q;
};

// u^_j is real and even in each component of k: M^g phit_j is a real function
// of |d| on the cyclic grid, so its DFT is the separable DCT-I of the octant
// d in [0,16]^3 (weights 1 at d = 0 and d = 16, 2 in between), stored for
// k in [0,16]^3 and read back through k -> min(k, 32 - k).
constexpr int U_N = 17, U_SZ = U_N * U_N * U_N;
constexpr int U_STRIDE = 4916;  // U_SZ rounded up to 16-byte rows
constexpr int U_THREADS = 320;

__device__ __forceinline__ int fold32(int i) { return i <= 16 ? i : 32 - i; }

// c_d cos(pi k d / 16) for k = 0..16, d = 0..7 (c_0 = 1, c_d = 2 otherwise).
// Pairing d with 16 - d (cos(pi k (16 - d) / 16) = (-1)^k cos(pi k d / 16))
// splits the length-17 DCT-I into 9 even outputs over x_d + x_(16-d) (plus
// the middle term 2 x_8 cos(pi k / 2)) and 8 odd outputs over x_d - x_(16-d).
static __constant__ float c_dct17[17 * 8];

static cudaError_t upload_dct() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  float t[17 * 8];
  for (int k = 0; k <= 16; ++k)
    for (int d = 0; d < 8; ++d)
      t[k * 8 + d] = (float)((d == 0 ? 1.0 : 2.0) * std::cos(3.14159265358979323846 * k * d / 16.0));
  e = cudaMemcpyToSymbol(c_dct17, t, sizeof(t));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

// y_k of the DCT-I of x, written to dst[k * stride] as soon as it is formed
__device__ __forceinline__ void dct17(const float (&x)[U_N], float* dst, int stride) {
  float ev[8], od[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) {
    ev[d] = x[d] + x[16 - d];
    od[d] = x[d] - x[16 - d];
  }
#pragma unroll
  for (int k = 0; k <= 16; ++k) {
    float acc = (k & 1) ? 0.f : ((k & 2) ? -2.f * x[8] : 2.f * x[8]);
#pragma unroll
    for (int d = 0; d < 8; ++d) acc = fmaf(c_dct17[k * 8 + d], (k & 1) ? od[d] : ev[d], acc);
    dst[k * stride] = acc;
  }
}

// Per-instance FP64 tables of a CTA.  With a_d(i) = (v_i - u_d)^2 rounded as
// in the definition, |v-u|^2 = (a_1 + a_2) + a_3 exactly as the oracle forms
// it; M = em_1 em_2 em_3 and 1/M = ei_1 ei_2 ei_3 (axis 1 carries the
// prefactors).  The cut-off of Eq. (3.9), fl(|v-u|^2 / (2 theta)) > thr, is
// monotone in |v-u|^2, so it is replaced by the exact equivalent
// |v-u|^2 >= dstar, dstar the smallest double that passes the test.
struct PrepTables {
  double a[3 * 32], em[3 * 32], ei[3 * 32];
  float eif[3 * 32];  // ei in FP32, for the ratio of the head kernel
  float emf[3 * 32];  // em in FP32, for the loss term
  double dstar;
};

__device__ __forceinline__ void fill_prep(PrepTables& T, const InstanceParams& q, double h, double log_inv_eps) {
  const int t = threadIdx.x;
  if (t < 96) {
    const int d = t / 32, i = t % 32;
    const double ud = d == 0 ? q.u1 : (d == 1 ? q.u2 : q.u3);
    const double dv = __dsub_rn(__dmul_rn((double)(i - 16), h), ud);
    const double a2 = __dmul_rn(dv, dv);
    T.a[t] = a2;
    double em = exp(-a2 / (2.0 * q.theta)), ei = exp(a2 / (2.0 * q.theta));
    if (d == 0) {
      const double pref = q.rho * pow(2.0 * 3.141592653589793 * q.theta, -1.5);
      em *= pref;
      ei /= pref;
    }
    T.em[t] = em;
    T.ei[t] = ei;
    T.eif[t] = (float)ei;
    T.emf[t] = (float)em;
  } else if (t == 96) {
    const double twoth = __dmul_rn(2.0, q.theta);
    const double thr = __dsub_rn(log_inv_eps, __dmul_rn(1.5, log(__dmul_rn(__dmul_rn(2.0, 3.141592653589793), q.theta))));
    double x = __dmul_rn(thr, twoth);
    for (int it = 0; it < 64 && __ddiv_rn(x, twoth) > thr; ++it) x = nextafter(x, -1e308);
    for (int it = 0; it < 64 && !(__ddiv_rn(x, twoth) > thr); ++it) x = nextafter(x, 1e308);
    T.dstar = x;
  }
  __syncthreads();
}

// rows (i1, q) of a real source -> forward half spectrum in V (all three axes
// except axis 1, which the caller fuses with its pointwise stage).
template <typename Src>
__device__ __forceinline__ void rows_forward(cpx<float>* V, Src src) {
  const int t = threadIdx.x;
  if (t < 512) {
    const int i1 = t >> 4, qq = t & 15;
    cpx<float> z[32];
#pragma unroll
    for (int i3 = 0; i3 < 32; ++i3) z[i3] = src(i1, qq, i3);
    fft32<false>(z);
    split_store(z, V + i1 * S_PLANE + qq * S_PAIR);
  }
  __syncthreads();
  axis_pass<2, false>(V);
  __syncthreads();
}

// r^ = FFT(r) / N^3, r = g/M with the cut-off of Eq. (3.9).
__global__ void __launch_bounds__(F_THREADS, 1) k_f32_head(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  __shared__ PrepTables T;
  const int b = blockIdx.x, t = threadIdx.x;
  const InstanceParams q = load_params(a.params, b);
  fill_prep(T, q, a.h, a.log_inv_eps);
  const double* gb = a.g + (size_t)b * 32768;
  const bool cut = a.cutoff != 0;
  // The cut-off decision stays in FP64 exactly as the oracle forms it,
  // ((a_1 + a_2) + a_3) >= d*, with the row sum a_1 + a_2 hoisted; the ratio
  // itself is formed in FP32 (it is rounded to FP32 for the transform
  // anyway).  A point that passes the cut has (a_1 + a_2) / (2 theta) below
  // the threshold, so its partial product stays finite; a cut point is
  // selected, never multiplied.  Without the cut-off the factors 1/M of the
  // outer points exceed the FP32 range (exp(|v-u|^2/(2 theta)) reaches
  // 1e94 on the box), so the ratio is then formed in FP64 and only r is
  // rounded to FP32.
  if (cut) {
    rows_forward(V, [&](int i1, int qq, int i3) {
      float v[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int i2 = 2 * qq + r;
        const double d2 = __dadd_rn(__dadd_rn(T.a[i1], T.a[32 + i2]), T.a[64 + i3]);
        const float val = (float)gb[(i1 * 32 + i2) * 32 + i3] * ((T.eif[i1] * T.eif[32 + i2]) * T.eif[64 + i3]);
        v[r] = d2 >= T.dstar ? 0.f : val;
      }
      return make_c(v[0], v[1]);
    });
  } else {
    rows_forward(V, [&](int i1, int qq, int i3) {
      float v[2];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int i2 = 2 * qq + r;
        v[r] = (float)(gb[(i1 * 32 + i2) * 32 + i3] * ((T.ei[i1] * T.ei[32 + i2]) * T.ei[64 + i3]));
      }
      return make_c(v[0], v[1]);
    });
  }
  const int i2 = t / F_HC, k3 = t % F_HC;
  cpx<float>* base = V + srow(i2) + k3;
  cpx<float> x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = base[i * S_PLANE];
  fft32<false>(x);
  cpx<float>* dst = a.rhat + (size_t)b * F_H + i2 * F_HC + k3;
  const float s = 1.0f / 32768.0f;
#pragma unroll
  for (int i = 0; i < 32; ++i) dst[i * F_ROW] = cscale(x[i], s);
}

// u^_j of instance b (block (j, b)): w(d) = rho (pi theta)^-3/2
// exp(-|d h|^2/theta) phit_j(d) on the octant, then the DCT-I along each axis.
__global__ void __launch_bounds__(U_THREADS, 4) k_f32_uhat(FusedArgs a) {
  __shared__ float W[U_SZ];
  __shared__ float mg[U_N + 1];  // mg[17] = rho (pi theta)^-3/2
  const int j = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
  if (t <= U_N) {
    const double rho = a.params[5 * b], theta = a.params[5 * b + 4];
    if (t < U_N) {
      const double x = t * a.h;
      mg[t] = (float)exp(-(x * x) / theta);
    } else {
      mg[U_N] = (float)(rho * pow(3.141592653589793 * theta, -1.5));
    }
  }
  __syncthreads();
  const float pref = mg[U_N];
  const float* ph = a.phit + (size_t)j * 32768;
  for (int e = t; e < U_SZ; e += U_THREADS) {
    const int d1 = e / (U_N * U_N), d2 = (e / U_N) % U_N, d3 = e % U_N;
    W[e] = pref * (mg[d1] * mg[d2]) * mg[d3] * __ldg(ph + (d1 * 32 + d2) * 32 + d3);
  }
  __syncthreads();
#pragma unroll 1
  for (int axis = 3; axis >= 1; --axis) {
    if (t < U_N * U_N) {
      const int p0 = t / U_N, p1 = t % U_N;
      // pencil start and stride along the transformed axis
      const int base = axis == 3 ? t * U_N : (axis == 2 ? p0 * U_N * U_N + p1 : t);
      const int stride = axis == 3 ? 1 : (axis == 2 ? U_N : U_N * U_N);
      float x[U_N];
#pragma unroll
      for (int d = 0; d < U_N; ++d) x[d] = W[base + d * stride];
      dct17(x, W + base, stride);
    }
    __syncthreads();
  }
  float* dst = a.uhat + ((size_t)b * a.J + j) * U_STRIDE;
  for (int e = t; e < U_SZ; e += U_THREADS) dst[e] = W[e];
}

// Loss term of one instance, lossf = -InvFFT(FFT(g) omega) M - InvFFT(FFT(M) omega) g (FP32).
__device__ void loss_term(const FusedArgs& a, cpx<float>* V, const PrepTables& T, int b) {
  const int t = threadIdx.x;
  const double* gb = a.g + (size_t)b * 32768;
  float* ob = a.lossf + (size_t)b * 32768;
  for (int pass = 0; pass < 2; ++pass) {
    rows_forward(V, [&](int i1, int qq, int i3) {
      if (pass == 0)
        return make_c((float)gb[(i1 * 32 + 2 * qq) * 32 + i3], (float)gb[(i1 * 32 + 2 * qq + 1) * 32 + i3]);
      const float m13 = T.emf[i1] * T.emf[64 + i3];
      return make_c(m13 * T.emf[32 + 2 * qq], m13 * T.emf[32 + 2 * qq + 1]);
    });
    {
      const int i2 = t / F_HC, k3 = t % F_HC;
      cpx<float>* base = V + srow(i2) + k3;
      cpx<float> x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = base[i * S_PLANE];
      fft32<false>(x);
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = cscale(x[i], __ldg(a.omega + ksq(i, i2, k3)));
      fft32<true>(x);
#pragma unroll
      for (int i = 0; i < 32; ++i) base[i * S_PLANE] = x[i];
    }
    __syncthreads();
    axis_pass<2, true>(V);
    __syncthreads();
    if (t < 512) {
      const int i1 = t >> 4, qq = t & 15;
      cpx<float> z[32];
      load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
      fft32<true>(z);
      // FP32: every term carries the rounding of an FP32 transform
      float* o0 = ob + (i1 * 32 + 2 * qq) * 32;
      const double* g0 = gb + (i1 * 32 + 2 * qq) * 32;
      const float ma = T.emf[i1] * T.emf[32 + 2 * qq], mb = T.emf[i1] * T.emf[32 + 2 * qq + 1];
#pragma unroll 4
      for (int i3 = 0; i3 < 32; ++i3) {
        if (pass == 0) {  // -u M
          o0[i3] = -z[i3].x * (ma * T.emf[64 + i3]);
          o0[32 + i3] = -z[i3].y * (mb * T.emf[64 + i3]);
        } else {  // -w g
          o0[i3] -= z[i3].x * (float)g0[i3];
          o0[32 + i3] -= z[i3].y * (float)g0[32 + i3];
        }
      }
    }
    __syncthreads();
  }
}

// u^_j of the next radial node is staged into shared memory by a bulk
// asynchronous copy (cp.async.bulk, 19664 bytes: both addresses 16-byte
// aligned, size a multiple of 16) while the current node runs, two buffers
// each with its mbarrier; every wait is bounded and sets a.err when it gives up.
constexpr uint32_t U_BYTES = U_STRIDE * sizeof(float);
static_assert(U_BYTES % 16 == 0, "bulk copy size");
constexpr size_t GAIN_SMEM = sizeof(cpx<float>) * S_TOTAL + 2 * U_BYTES;
constexpr uint32_t kUPolls = 1u << 22;

// (no memory clobber: the copy's data becomes visible through the bounded
// mbarrier wait, which carries one)
__device__ __forceinline__ void stage_uhat(uint32_t dst, const float* src, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(U_BYTES));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(U_BYTES), "r"(bar));
}

// The gain blocks hold the running partial L^+ in tensor memory: thread t
// owns the same pencil (i2, k3) = (t / 17, t % 17) in the first and the last
// pass of every j, so its 32 complex sums stay in 64 TMEM columns of its
// lane (warp w: lanes 32 (w % 4) + lane, columns 64 (w / 4) .. + 63; 17
// warps use 320 of the 512 columns) instead of a read-modify-write of the
// global partial per j.  The last j adds and writes the partial to global
// memory.  The dynamic shared memory keeps one such block per SM (two would
// need more than the SM's 228 KB), so the 512-column allocation never waits.
static_assert(2 * sizeof(cpx<float>) * S_TOTAL > 228 * 1024, "gain blocks must not share an SM");
static_assert(GAIN_SMEM + 8 * 1024 <= 227 * 1024, "gain block shared memory");
static_assert(64 * ((F_THREADS / 32 + 3) / 4) <= tmem::kColumns, "partial sums exceed TMEM");

// grid (G + 1, B): blocks x < G run the gain term for their group of radial
// nodes (partial L^+ = sum_j phi_j FFT(M^h InvFFT(u^_j r^))); block x = G
// writes the loss term of the instance into out.
__global__ void __launch_bounds__(F_THREADS, 1) k_f32_gain(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  float* ubuf = (float*)(smem + sizeof(cpx<float>) * S_TOTAL);  // [2][U_STRIDE]
  __shared__ float mh[3 * F_N];
  __shared__ PrepTables T;
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t ubar[2];
  const int grp = blockIdx.x, b = blockIdx.y, t = threadIdx.x;
  const InstanceParams q = load_params(a.params, b);
  if (grp == a.G) {
    fill_prep(T, q, a.h, a.log_inv_eps);
    loss_term(a, V, T, b);
    return;
  }
  const int j0 = (a.J * grp) / a.G, j1 = (a.J * (grp + 1)) / a.G;
  const float* usrc = a.uhat + (size_t)b * a.J * U_STRIDE;
  const uint32_t ubuf_s = umma::smem_u32(ubuf), bar0 = umma::smem_u32(&ubar[0]);
  if (t == 0) {
    umma::mbar_init(bar0, 1);
    umma::mbar_init(bar0 + 8, 1);
  }
  if (t < 32) tmem::alloc(&tmem_slot, tmem::kColumns);
  if (t < 3 * F_N) {
    int dd = t / F_N, i = t % F_N;
    double ud = dd == 0 ? q.u1 : (dd == 1 ? q.u2 : q.u3);
    double v = (double)(i - 16) * a.h - ud;
    double e = exp(-(v * v) / q.theta);
    if (dd == 0) e *= q.rho * pow(3.141592653589793 * q.theta, -1.5);
    mh[t] = (float)e;
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const uint32_t tbase = tmem_slot;
  const uint32_t tacc = tmem::addr(tbase, 32u * ((t >> 5) & 3), 64u * (t >> 7));
  const cpx<float>* rh = a.rhat + (size_t)b * F_H;
  cpx<float>* acc = a.part + ((size_t)grp * a.B + b) * F_H;
  for (int j = j0; j < j1; ++j) {
    const int slot = (j - j0) & 1;
    if (t == 0) {
      if (j == j0) stage_uhat(ubuf_s, usrc + (size_t)j0 * U_STRIDE, bar0);
      if (j + 1 < j1) {
        // the other buffer was last read by the first pass of node j - 1,
        // which every thread has left (several barriers ago)
        umma::fence_proxy_async_smem();
        stage_uhat(ubuf_s + (uint32_t)(slot ^ 1) * U_BYTES, usrc + (size_t)(j + 1) * U_STRIDE, bar0 + 8u * (slot ^ 1));
      }
    }
    if (!umma::mbar_wait_bounded(bar0 + 8u * slot, ((j - j0) >> 1) & 1, kUPolls)) atomicExch(a.err, 1);
    {  // axis 1: psi^_j = u^_j r^ (r^ pre-scaled), inverse
      const int i2 = t / F_HC, k3 = t % F_HC;
      cpx<float>* base = V + srow(i2) + k3;
      const cpx<float>* rr = rh + i2 * F_HC + k3;
      const float* uk = ubuf + slot * U_STRIDE + fold32(i2) * U_N + k3;
      cpx<float> x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = cscale(rr[i * F_ROW], uk[fold32(i) * (U_N * U_N)]);
      fft32<true>(x);
#pragma unroll
      for (int i = 0; i < 32; ++i) base[i * S_PLANE] = x[i];
    }
    __syncthreads();
    axis_pass<2, true>(V);
    __syncthreads();
    if (t < 512) {  // rows: inverse, x M^h, forward
      const int i1 = t >> 4, qq = t & 15;
      cpx<float>* row = V + i1 * S_PLANE + qq * S_PAIR;
      cpx<float> z[32];
      load_merge(row, z);
      fft32<true>(z);
      const float m1 = mh[i1], ma = m1 * mh[F_N + 2 * qq], mb = m1 * mh[F_N + 2 * qq + 1];
#pragma unroll
      for (int i3 = 0; i3 < 32; ++i3) {
        const float m3 = mh[2 * F_N + i3];
        z[i3] = make_c(z[i3].x * (ma * m3), z[i3].y * (mb * m3));
      }
      fft32<false>(z);
      split_store(z, row);
    }
    __syncthreads();
    axis_pass<2, false>(V);
    __syncthreads();
    {  // axis 1 forward, accumulate phi_j(|k|^2) psi^_j (TMEM; global at the last j)
      const int i2 = t / F_HC, k3 = t % F_HC;
      cpx<float>* base = V + srow(i2) + k3;
      cpx<float>* ac = acc + i2 * F_HC + k3;
      const float* ph = a.phi + (size_t)j * a.Q;
      const bool first = j == j0, last = j + 1 == j1;
      cpx<float> x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = base[i * S_PLANE];
      fft32<false>(x);
#pragma unroll
      for (int c = 0; c < 8; ++c) {  // 4 complex sums = 8 columns per chunk
        uint32_t r[8];
        if (!first) {
          tmem::ld8(tacc + 8 * c, r);
          tmem::wait_ld(r);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * c + e;
          cpx<float> v = cscale(x[i], __ldg(ph + ksq(i, i2, k3)));
          if (!first) v = make_c(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1])) + v;
          if (last) {
            ac[i * F_ROW] = v;
          } else {
            r[2 * e] = __float_as_uint(v.x);
            r[2 * e + 1] = __float_as_uint(v.y);
          }
        }
        if (!last) tmem::st8(tacc + 8 * c, r);
      }
      if (!last) tmem::wait_st();
    }
    // no barrier before the next node: its first pass writes, thread by
    // thread, the same pencil this thread has just read (axis-1 pencils
    // are private to their thread in the first and the last pass), and the
    // partial sums and r^ are private to the thread as well
  }
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  if (t == 0) {
    // no copy is left in flight when every wait succeeded; after a timeout,
    // one more bounded wait on the last phase of each buffer
    const int n = j1 - j0;
    for (int sl = 0; sl < 2 && sl < n; ++sl) {
      const int uses = (n - sl + 1) / 2;
      umma::mbar_wait_bounded(bar0 + 8u * sl, (uses - 1) & 1, kUPolls);
    }
  }
  if (t < 32) tmem::dealloc(tbase, tmem::kColumns);
}

// out = InvFFT(sum over groups of the partial L^+) + the loss term, in FP64.
__global__ void __launch_bounds__(F_THREADS, 1) k_f32_tail(FusedArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cpx<float>* V = (cpx<float>*)smem;
  const int b = blockIdx.x, t = threadIdx.x;
  {
    const int i2 = t / F_HC, k3 = t % F_HC;
    cpx<float> x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = make_c(0.f, 0.f);
    for (int gi = 0; gi < a.G; ++gi) {
      const cpx<float>* src = a.part + ((size_t)gi * a.B + b) * F_H + i2 * F_HC + k3;
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = x[i] + src[i * F_ROW];
    }
    fft32<true>(x);
    cpx<float>* base = V + srow(i2) + k3;
#pragma unroll
    for (int i = 0; i < 32; ++i) base[i * S_PLANE] = x[i];
  }
  __syncthreads();
  axis_pass<2, true>(V);
  __syncthreads();
  if (t < 512) {
    const int i1 = t >> 4, qq = t & 15;
    cpx<float> z[32];
    load_merge(V + i1 * S_PLANE + qq * S_PAIR, z);
    fft32<true>(z);
    double* o0 = a.out + (size_t)b * 32768 + (i1 * 32 + 2 * qq) * 32;
    const float* l0 = a.lossf + (size_t)b * 32768 + (i1 * 32 + 2 * qq) * 32;
#pragma unroll
    for (int i3 = 0; i3 < 32; ++i3) {  // out = L+ + loss, summed in FP32
      o0[i3] = (double)(z[i3].x + l0[i3]);
      o0[32 + i3] = (double)(z[i3].y + l0[32 + i3]);
    }
  }
}

}  // namespace

size_t fused32_workspace_bytes(int B, int G, int J) {
  return (size_t)B * F_H * 8 * (1 + (size_t)G) + (size_t)B * J * U_STRIDE * sizeof(float) +
         (size_t)B * 32768 * sizeof(float);
}

int fused32_default_groups(int B) {
  // enough CTAs to fill 152 SMs several times over, at most 8 groups
  int g = (4 * 152 + B - 1) / B;
  return g < 1 ? 1 : (g > 8 ? 8 : g);
}

size_t fused32_uhat_bytes(int B, int J) { return (size_t)B * J * U_STRIDE * sizeof(float); }

// u^_j of every instance and radial node into uhat ([B][J][U_STRIDE]), for
// the Maxwellian cache: k_f32_uhat alone.
lbo_status precompute_fused32(lbo_plan* p, const double* params, int B, float* uhat) {
  cudaError_t e = upload_twiddles();
  if (e == cudaSuccess) e = upload_dct();
  if (e != cudaSuccess) return cuda_fail(e, "fused32 twiddles");
  FusedArgs a{};
  a.params = params;
  a.phit = p->d_phit32;
  a.uhat = uhat;
  a.h = 2.0 * p->L / F_N;
  a.J = p->J;
  a.B = B;
  LBO_LAUNCH(p, "cache_f32_uhat", p->stream, k_f32_uhat, dim3(a.J, B), U_THREADS, 0, a);
  p->last_launches = 1;
  e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "fused32 cache launch");
}

lbo_status run_linearized_fused32(lbo_plan* p, const double* params, const double* g, double* out, int B,
                                  void* ws, int G, int* launches, const float* cached_uhat) {
  cudaError_t e = upload_twiddles();
  if (e == cudaSuccess) e = upload_dct();
  if (e != cudaSuccess) return cuda_fail(e, "fused32 twiddles");
  const size_t sm = sizeof(cpx<float>) * S_TOTAL;
  raise_smem_limit((const void*)k_f32_head, sm);
  raise_smem_limit((const void*)k_f32_gain, GAIN_SMEM);
  raise_smem_limit((const void*)k_f32_tail, sm);
  if (!p->d_tc_err) {
    e = cudaMalloc(&p->d_tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_tc_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait error flag");
  }
  FusedArgs a{};
  a.params = params;
  a.g = g;
  a.phit = p->d_phit32;
  a.phi = p->d_phi32;
  a.omega = p->d_omega32;
  a.rhat = (cpx<float>*)ws;
  a.part = a.rhat + (size_t)B * F_H;
  a.uhat = (float*)(a.part + (size_t)G * B * F_H);
  a.lossf = a.uhat + (size_t)B * p->J * U_STRIDE;
  a.out = out;
  a.err = (int*)p->d_tc_err;
  a.h = 2.0 * p->L / F_N;
  a.log_inv_eps = std::log(1.0 / p->eps);
  a.cutoff = p->cutoff;
  a.J = p->J;
  a.G = G;
  a.B = B;
  a.Q = 3 * 16 * 16 + 1;
  cudaStream_t s = p->stream;
  LBO_LAUNCH(p, "f32_head", s, k_f32_head, B, F_THREADS, sm, a);
  if (cached_uhat) {
    a.uhat = const_cast<float*>(cached_uhat);  // read only from here on
  } else {
    LBO_LAUNCH(p, "f32_uhat", s, k_f32_uhat, dim3(a.J, B), U_THREADS, 0, a);
    *launches += 1;
  }
  LBO_LAUNCH(p, "f32_gain", s, k_f32_gain, dim3(G + 1, B), F_THREADS, GAIN_SMEM, a);
  LBO_LAUNCH(p, "f32_tail", s, k_f32_tail, B, F_THREADS, sm, a);
  *launches += 3;
  e = cudaGetLastError();
  return e == cudaSuccess ? LBO_OK : cuda_fail(e, "fused32 launch");
}

}  // namespace lbo

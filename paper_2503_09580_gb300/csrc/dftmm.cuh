// One axis pass of a batched 3-D DFT as a dense contraction on the
// tensor cores (tcgen05.mma, kind::f16, FP32 accumulation in TMEM), with
// split 16-bit operands: x = x_hi + x_lo, W = W_hi + W_lo (each part
// rounded to BF16 or FP16) and W x ~ W_hi x_hi + W_lo x_hi + W_hi x_lo, three
// products per K-slice (the dropped W_lo x_lo is ~2^-16 (BF16) or ~2^-22
// (FP16) of the product).
//
// A complex pencil of length N is a row of 2N reals (re, im interleaved);
// the length-N DFT is the real (2N x 2N) matrix W with rows 2q (real part of
// output q) and 2q + 1 (imaginary part):
//     W[2q][2j] = a, W[2q][2j+1] = -b, W[2q+1][2j] = b, W[2q+1][2j+1] = a,
// a + i b the complex DFT entry.  One CTA of 128 threads takes 128 pencils
// per tile (thread t owns pencil t: it loads, splits and writes row t of the
// A operand, then reads row t of D = A W^T from TMEM lane t): M = 128,
// N = K = 2N.  W stays in shared memory for the whole (persistent) kernel.
//
// Index conventions: a real-space axis is in the library's centred order
// (index i <-> l = i - N/2), a frequency axis in cyclic order (k = 0..N-1);
// forward W[q][j] = exp(-2 pi i q (j - N/2) / N), inverse
// W[j][q] = exp(+2 pi i q (j - N/2) / N), unnormalised.
//
// FP16 operands carry 11 bits each but only 5 exponent bits: every pencil
// is scaled by a power of two (max |x| 2^-e in [0.5, 1)) before the split
// and the scale is undone on D.  BF16 has the FP32 exponent range and is not
// scaled.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "lin_kernels.cuh"
#include "tmem.cuh"
#include "umma.cuh"

namespace lbo {
namespace mm {

constexpr int kTile = 128;           // pencils per tile (the MMA's M)
constexpr uint32_t kMaxPolls = 1u << 22;  // bounded wait on an MMA completion

// Pointwise stage before the transform (on the element at its full index).
enum Pre {
  PRE_NONE = 0,
  PRE_RATIO = 1,   // r = g / M (0 where the cut-off of Eq. (3.9) applies), from FP64 g; real space
  PRE_REAL64 = 2,  // the FP64 field g; real space
  PRE_UHAT = 3,    // x u^_j(|k1|, |k2|, k3) scale (cached octant); frequency space
  PRE_MH = 4       // Re(x) M^h(v); real space
};
// Stage after the transform.
enum Post {
  POST_STORE = 0,   // dst = y
  POST_ACC = 1,     // dst (+)= table(|k|^2) y (first: store)
  POST_REAL = 2,    // dst = (Re y, 0)
  POST_REAL64 = 3,  // dst64 = Re y (FP64)
  POST_TABLE = 4    // dst = table(|k|^2) y
};

struct PassArgs {
  const float2* src;     // [B][N^3] complex (not read by PRE_RATIO / PRE_REAL64)
  float2* dst;           // [B][N^3] complex (may equal src)
  double* dst64;         // [B][N^3] real (POST_REAL64)
  const double* params;  // [B][5]
  const double* g;       // [B][N^3] FP64 (PRE_RATIO, PRE_REAL64)
  const float* uhat;     // [B][(N/2+1)^3] octant of u^_j (PRE_UHAT)
  const float* table;    // [3(N/2)^2+1] by |k|^2 (POST_ACC, POST_TABLE)
  const uint16_t* wmat;  // W_hi then W_lo in the shared-memory image (umma.cuh layout)
  int* err;              // set to 1 when an MMA completion wait gives up
  double h, log_inv_eps;
  float scale;           // PRE_UHAT
  int cutoff, first, B;
};

template <int N>
struct Geo {
  static constexpr int K = 2 * N;                        // reals per pencil
  static constexpr int ROW_BYTES = K * 2;                // one 16-bit row
  static constexpr int W_BYTES = K * K * 2;              // one part of W
  static constexpr int A_BYTES = kTile * K * 2;          // one part of A
  static constexpr int SMEM = 2 * W_BYTES + 2 * A_BYTES;  // W hi, lo; A hi, lo
  static constexpr int TMEM_COLS = K < 32 ? 32 : K;      // D: 128 lanes x K FP32 columns
  static constexpr int HC = N / 2 + 1;
};

// element offset of (pencil P, position j) along AXIS (1, 2, 3 = i1, i2, i3)
template <int N, int AXIS>
__device__ __forceinline__ size_t elem(size_t P, int j) {
  const size_t b = P / (N * N), r = P % (N * N);
  if constexpr (AXIS == 3) return P * N + j;                                         // r = i1 N + i2
  else if constexpr (AXIS == 2) return (b * N + r / N) * N * N + (size_t)j * N + r % N;  // r = i1 N + i3
  else return b * (size_t)N * N * N + (size_t)j * N * N + r;                          // r = i2 N + i3
}

// the three indices of (pencil P, position j)
template <int N, int AXIS>
__device__ __forceinline__ void index3(size_t P, int j, int& i1, int& i2, int& i3) {
  const int r = (int)(P % (N * N));
  if constexpr (AXIS == 3) { i1 = r / N; i2 = r % N; i3 = j; }
  else if constexpr (AXIS == 2) { i1 = r / N; i2 = j; i3 = r % N; }
  else { i1 = j; i2 = r / N; i3 = r % N; }
}

template <int N>
__device__ __forceinline__ int absfreq(int k) { return k <= N / 2 ? k : N - k; }

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b, float s, uint32_t& lo) {
  if constexpr (BF) {
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
    return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
  } else {
    a *= s;
    b *= s;
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    const __half la = __float2half_rn(a - __half2float(ha)), lb = __float2half_rn(b - __half2float(hb));
    lo = (uint32_t)__half_as_ushort(la) | ((uint32_t)__half_as_ushort(lb) << 16);
    return (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
  }
}

// Per-instance FP64 tables of a tile (its 128 pencils lie in one instance):
// a = (v_i - u_d)^2, em = exp(-a/(2 theta)) (axis 1 times the prefactor),
// ei = 1/em, eh = the factors of M^h; dstar: the smallest |v-u|^2 that the
// cut-off of Eq. (3.9) zeroes, fl(|v-u|^2/(2 theta)) > thr, found by
// stepping ulps (the test is monotone in |v-u|^2).
template <int N>
struct InstTables {
  double a[3 * N], em[3 * N], ei[3 * N];
  float eif[3 * N], ehf[3 * N];  // 1/M and M^h factors in FP32 (the operands are 16-bit)
  double dstar;
  int b;
};

template <int N>
__device__ void fill_inst(InstTables<N>& T, const double* params, int b, double h, double log_inv_eps) {
  const InstanceParams q = load_params(params, b);
  for (int t = threadIdx.x; t < 3 * N; t += blockDim.x) {
    const int d = t / N, i = t % N;
    const double ud = d == 0 ? q.u1 : (d == 1 ? q.u2 : q.u3);
    const double dv = __dsub_rn(__dmul_rn((double)(i - N / 2), h), ud);
    const double a2 = __dmul_rn(dv, dv);
    T.a[t] = a2;
    double em = exp(-a2 / (2.0 * q.theta)), ei = exp(a2 / (2.0 * q.theta)), eh = exp(-a2 / q.theta);
    if (d == 0) {
      const double pref = q.rho * pow(2.0 * 3.141592653589793 * q.theta, -1.5);
      em *= pref;
      ei /= pref;
      eh *= q.rho * pow(3.141592653589793 * q.theta, -1.5);
    }
    T.em[t] = em;
    T.ei[t] = ei;
    T.eif[t] = (float)ei;
    T.ehf[t] = (float)eh;
  }
  if (threadIdx.x == 0) {
    const double twoth = __dmul_rn(2.0, q.theta);
    const double thr =
        __dsub_rn(log_inv_eps, __dmul_rn(1.5, log(__dmul_rn(__dmul_rn(2.0, 3.141592653589793), q.theta))));
    double x = __dmul_rn(thr, twoth);
    for (int it = 0; it < 64 && __ddiv_rn(x, twoth) > thr; ++it) x = nextafter(x, -1e308);
    for (int it = 0; it < 64 && !(__ddiv_rn(x, twoth) > thr); ++it) x = nextafter(x, 1e308);
    T.dstar = x;
    T.b = b;
  }
}

template <int N, int AXIS, int PRE>
__device__ __forceinline__ float2 load_pre(const PassArgs& a, const InstTables<N>& T, size_t P, int j) {
  int i1, i2, i3;
  index3<N, AXIS>(P, j, i1, i2, i3);
  const size_t b = P / (N * N);
  const size_t e = elem<N, AXIS>(P, j);
  if constexpr (PRE == PRE_RATIO) {
    if (a.cutoff) {
      // the cut-off decision in FP64 exactly as the oracle forms it; a point
      // that passes has |v-u|^2/(2 theta) below the threshold, so the FP32
      // product of its 1/M factors stays finite
      const double d2 = __dadd_rn(__dadd_rn(T.a[i1], T.a[N + i2]), T.a[2 * N + i3]);
      if (d2 >= T.dstar) return make_float2(0.f, 0.f);
      return make_float2((float)a.g[e] * ((T.eif[i1] * T.eif[N + i2]) * T.eif[2 * N + i3]), 0.f);
    }
    return make_float2((float)(a.g[e] * ((T.ei[i1] * T.ei[N + i2]) * T.ei[2 * N + i3])), 0.f);
  } else if constexpr (PRE == PRE_REAL64) {
    return make_float2((float)a.g[e], 0.f);
  } else {
    float2 x = a.src[e];
    if constexpr (PRE == PRE_UHAT) {
      constexpr int HC = N / 2 + 1;
      const float u = a.uhat[b * HC * HC * HC + ((size_t)absfreq<N>(i1) * HC + absfreq<N>(i2)) * HC + absfreq<N>(i3)];
      const float s = u * a.scale;
      x.x *= s;
      x.y *= s;
    } else if constexpr (PRE == PRE_MH) {
      x.x *= (T.ehf[i1] * T.ehf[N + i2]) * T.ehf[2 * N + i3];
      x.y = 0.f;
    }
    return x;
  }
}

template <int N>
__device__ __forceinline__ int ksq(int i1, int i2, int i3) {
  const int a = i1 <= N / 2 ? i1 : i1 - N, b = i2 <= N / 2 ? i2 : i2 - N, c = i3 <= N / 2 ? i3 : i3 - N;
  return a * a + b * b + c * c;
}

template <int N, int AXIS, int PRE, int POST, bool BF>
__global__ void __launch_bounds__(kTile) k_dft_pass(PassArgs a) {
  using G = Geo<N>;
  constexpr int K = G::K;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* w_hi = smem;
  unsigned char* w_lo = smem + G::W_BYTES;
  unsigned char* a_hi = smem + 2 * G::W_BYTES;
  unsigned char* a_lo = a_hi + G::A_BYTES;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ InstTables<N> T;
  const int t = threadIdx.x, warp = t >> 5;
  // W into shared memory (its image is already in the operand layout)
  {
    const uint4* src = (const uint4*)a.wmat;
    uint4* dst = (uint4*)smem;
    for (int i = t; i < 2 * G::W_BYTES / 16; i += kTile) dst[i] = src[i];
  }
  if (warp == 0) tmem::alloc(&tmem_slot, G::TMEM_COLS);
  if (t == 0) {
    umma::mbar_init(umma::smem_u32(&bar), 1);
    T.b = -1;
  }
  umma::fence_proxy_async_smem();
  tmem::fence_before_sync();
  __syncthreads();
  tmem::fence_after_sync();
  const uint32_t d_tmem = tmem_slot;
  const uint32_t bar_a = umma::smem_u32(&bar);
  const uint32_t idesc = umma::idesc_f16(kTile, K, BF);
  const uint32_t sbo = 16u * K;
  const size_t tiles = (size_t)a.B * N * N / kTile;
  uint32_t phase = 0;
  bool failed = false;
  for (size_t tile = blockIdx.x; tile < tiles && !failed; tile += gridDim.x) {
    const size_t P = tile * kTile + t;
    constexpr bool NEED_INST = PRE == PRE_RATIO || PRE == PRE_MH;
    if constexpr (NEED_INST) {
      const int b = (int)(tile * kTile / (N * N));
      if (b != T.b) {  // uniform over the CTA
        __syncthreads();
        fill_inst<N>(T, a.params, b, a.h, a.log_inv_eps);
        __syncthreads();
      }
    }
    // ---- A operand: row t = pencil P, split into hi and lo parts
    float s = 1.f;
    if constexpr (!BF) {
      float mx = 0.f;
      for (int j = 0; j < N; ++j) {
        const float2 x = load_pre<N, AXIS, PRE>(a, T, P, j);
        mx = fmaxf(mx, fmaxf(fabsf(x.x), fabsf(x.y)));
      }
      int e = 0;
      if (mx > 0.f) frexpf(mx, &e);
      // max |x| s in [0.5, 1); a pencil whose largest value is subnormal (M^h
      // underflows at the box corners) keeps s <= 2^125, so s and 1/s stay finite
      s = ldexpf(1.f, -max(e, -125));
    }
    for (int j0 = 0; j0 < N; j0 += 4) {  // 8 reals = one 16-byte row of a core matrix
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 x = load_pre<N, AXIS, PRE>(a, T, P, j0 + u);
        hi[u] = pack2<BF>(x.x, x.y, s, lo[u]);
      }
      const uint32_t off = umma::kmajor_offset(t, 2 * j0, K);
      *(uint4*)(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *(uint4*)(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    umma::fence_proxy_async_smem();
    tmem::fence_before_sync();
    __syncthreads();
    // ---- D = A_hi W_hi^T + A_hi W_lo^T + A_lo W_hi^T, one thread issues
    if (t == 0) {
      tmem::fence_after_sync();
      const uint32_t ah = umma::smem_u32(a_hi), al = umma::smem_u32(a_lo);
      const uint32_t wh = umma::smem_u32(w_hi), wl = umma::smem_u32(w_lo);
#pragma unroll
      for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t o = 256u * ks;
        umma::mma_f16(d_tmem, umma::sdesc(ah + o, 128, sbo), umma::sdesc(wh + o, 128, sbo), idesc, ks > 0);
        umma::mma_f16(d_tmem, umma::sdesc(ah + o, 128, sbo), umma::sdesc(wl + o, 128, sbo), idesc, 1);
        umma::mma_f16(d_tmem, umma::sdesc(al + o, 128, sbo), umma::sdesc(wh + o, 128, sbo), idesc, 1);
      }
      umma::commit(bar_a);
    }
    // one decision for the whole CTA, so that every thread leaves together
    const bool done = umma::mbar_wait_bounded(bar_a, phase, kMaxPolls);
    if (__syncthreads_or(!done)) {
      failed = true;
      if (t == 0) atomicExch(a.err, 1);
      break;
    }
    phase ^= 1;
    tmem::fence_after_sync();
    // ---- D row t -> the pointwise stage -> global
    const float inv_s = 1.f / s;
    const uint32_t lane_addr = d_tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < K; c0 += 32) {
      float v[32];
      umma::ld32(lane_addr + c0, v);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int q = c0 / 2 + u;
        float2 y = make_float2(v[2 * u] * inv_s, v[2 * u + 1] * inv_s);
        const size_t e = elem<N, AXIS>(P, q);
        if constexpr (POST == POST_STORE) {
          a.dst[e] = y;
        } else if constexpr (POST == POST_REAL) {
          a.dst[e] = make_float2(y.x, 0.f);
        } else if constexpr (POST == POST_REAL64) {
          a.dst64[e] = (double)y.x;
        } else {
          int i1, i2, i3;
          index3<N, AXIS>(P, q, i1, i2, i3);
          const float w = a.table[ksq<N>(i1, i2, i3)];
          y.x *= w;
          y.y *= w;
          if constexpr (POST == POST_ACC) {
            if (!a.first) {
              const float2 o = a.dst[e];
              y.x += o.x;
              y.y += o.y;
            }
          }
          a.dst[e] = y;
        }
      }
    }
    tmem::fence_before_sync();
    __syncthreads();
  }
  if (failed) {
    // give the MMA that did not complete a second bounded chance before the
    // allocation is released
    umma::mbar_wait_bounded(bar_a, phase, kMaxPolls);
  }
  tmem::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tmem::fence_after_sync();
    tmem::dealloc(tmem_slot, G::TMEM_COLS);
  }
}

}  // namespace mm
}  // namespace lbo

// Small batched FFT building blocks for N = 16, 24, 32, 48, 64 (sm_103a).
//
// A length-N transform (N = R1*R2) is done in place on pencils held in
// shared memory, in two in-place stages:
//   stage A: for each n1 < R1, an R2-point DFT over x[n1 + R1*n2], then the
//            twiddle W_N^{n1 k2}, written back to positions n1 + R1*k2;
//   stage B: for each k2 < R2, an R1-point DFT over positions n1 + R1*k2.
// The forward output is in digit-reversed order: position p = k1 + R1*k2
// holds frequency k = k2 + R2*k1.  The inverse runs the two stages
// backwards (stage B^-1 then stage A^-1 with conjugate twiddles) and takes
// digit-reversed input to natural output, so every stage is in place and
// needs no extra buffer.  Inverse transforms are unnormalised.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "twiddles_hi.h"
#include "twofold.cuh"

namespace lbo {

template <typename T>
struct cpx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> make_c(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return make_c(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return make_c(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return make_c(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {  // a * conj(b)
  return make_c(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return make_c(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ cpx<T> conjc(cpx<T> a) { return make_c(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV>
__device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) {
  return INV ? make_c(-a.y, a.x) : make_c(a.y, -a.x);
}

// W_64^m = exp(-2 pi i m / 64), m = 0..63, and W_48^m (radix-3 sizes N = 24,
// 48), in every transform precision: double, float, and the two-fold pairs
// {re.hi, re.lo, im.hi, im.lo}.  Each translation unit has its own copy (no
// relocatable device code); upload_twiddles() fills it once per device from
// the double-pair table of twiddles_hi.h.
static __constant__ double2 c_tw64_d[64];
static __constant__ float2 c_tw64_f[64];
static __constant__ float4 c_tw64_ff[64];
static __constant__ double2 c_tw64_dd[2 * 64];  // [2m] = (re.hi, re.lo), [2m+1] = (im.hi, im.lo)
static __constant__ double2 c_tw48_d[48];
static __constant__ float2 c_tw48_f[48];
static __constant__ float4 c_tw48_ff[48];
static __constant__ double2 c_tw48_dd[2 * 48];

// a double pair (hi, lo) as a float pair carrying ~48 bits
static inline void split_to_float_pair(double hi, double lo, float* fh, float* fl) {
  *fh = (float)hi;
  *fl = (float)((hi - (double)*fh) + lo);
}

template <int NT>
static void fill_tw(const double (*src)[4], double2* d, float2* f, float4* ff, double2* dd) {
  for (int m = 0; m < NT; ++m) {
    d[m] = make_double2(src[m][0], src[m][2]);
    f[m] = make_float2((float)src[m][0], (float)src[m][2]);
    float a, b, c, e;
    split_to_float_pair(src[m][0], src[m][1], &a, &b);
    split_to_float_pair(src[m][2], src[m][3], &c, &e);
    ff[m] = make_float4(a, b, c, e);
    dd[2 * m] = make_double2(src[m][0], src[m][1]);
    dd[2 * m + 1] = make_double2(src[m][2], src[m][3]);
  }
}

static cudaError_t upload_twiddles_now() {
  double2 d[64], d48[48], dd[128], dd48[96];
  float2 f[64], f48[48];
  float4 ff[64], ff48[48];
  fill_tw<64>(kTw64Hi, d, f, ff, dd);
  fill_tw<48>(kTw48Hi, d48, f48, ff48, dd48);
  cudaError_t e = cudaMemcpyToSymbol(c_tw64_d, d, sizeof(d));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw64_f, f, sizeof(f));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw64_ff, ff, sizeof(ff));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw64_dd, dd, sizeof(dd));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw48_d, d48, sizeof(d48));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw48_f, f48, sizeof(f48));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw48_ff, ff48, sizeof(ff48));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_tw48_dd, dd48, sizeof(dd48));
  return e;
}

// Uploads this translation unit's tables once per device.
static cudaError_t upload_twiddles() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = upload_twiddles_now();
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

template <typename T>
__device__ __forceinline__ cpx<T> tw64(int m);
template <>
__device__ __forceinline__ cpx<double> tw64<double>(int m) {
  double2 t = c_tw64_d[m & 63];
  return make_c(t.x, t.y);
}
template <>
__device__ __forceinline__ cpx<float> tw64<float>(int m) {
  float2 t = c_tw64_f[m & 63];
  return make_c(t.x, t.y);
}

template <>
__device__ __forceinline__ cpx<f32x2> tw64<f32x2>(int m) {
  float4 t = c_tw64_ff[m & 63];
  return make_c(f32x2(t.x, t.y), f32x2(t.z, t.w));
}
template <>
__device__ __forceinline__ cpx<f64x2> tw64<f64x2>(int m) {
  double2 a = c_tw64_dd[2 * (m & 63)], b = c_tw64_dd[2 * (m & 63) + 1];
  return make_c(f64x2(a.x, a.y), f64x2(b.x, b.y));
}

template <typename T>
__device__ __forceinline__ cpx<T> tw48(int m);
template <>
__device__ __forceinline__ cpx<double> tw48<double>(int m) {
  double2 t = c_tw48_d[m % 48];
  return make_c(t.x, t.y);
}
template <>
__device__ __forceinline__ cpx<float> tw48<float>(int m) {
  float2 t = c_tw48_f[m % 48];
  return make_c(t.x, t.y);
}
template <>
__device__ __forceinline__ cpx<f32x2> tw48<f32x2>(int m) {
  float4 t = c_tw48_ff[m % 48];
  return make_c(f32x2(t.x, t.y), f32x2(t.z, t.w));
}
template <>
__device__ __forceinline__ cpx<f64x2> tw48<f64x2>(int m) {
  double2 a = c_tw48_dd[2 * (m % 48)], b = c_tw48_dd[2 * (m % 48) + 1];
  return make_c(f64x2(a.x, a.y), f64x2(b.x, b.y));
}

// W_N^m for N dividing 64 or 48
template <typename T, int N>
__device__ __forceinline__ cpx<T> twN(int m) {
  if constexpr (64 % N == 0) return tw64<T>((64 / N) * m);
  else return tw48<T>((48 / N) * m);
}

// ----------------------------------------------------------- small DFTs
template <typename T, bool INV>
__device__ __forceinline__ void dft2(cpx<T>* a) {
  cpx<T> t = a[0];
  a[0] = t + a[1];
  a[1] = t - a[1];
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cpx<T>* a) {
  cpx<T> t0 = a[0] + a[2], t1 = a[0] - a[2];
  cpx<T> t2 = a[1] + a[3], t3 = mul_mi<T, INV>(a[1] - a[3]);
  a[0] = t0 + t2;
  a[2] = t0 - t2;
  a[1] = t1 + t3;
  a[3] = t1 - t3;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft8(cpx<T>* a) {
  const T r = kconst<T>(0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55);  // 1/sqrt2
  cpx<T> e[4] = {a[0], a[2], a[4], a[6]};
  cpx<T> o[4] = {a[1], a[3], a[5], a[7]};
  dft4<T, INV>(e);
  dft4<T, INV>(o);
  // W8^1 = (1 -+ i)/sqrt2, W8^2 = -+i, W8^3 = (-1 -+ i)/sqrt2
  cpx<T> o1 = INV ? make_c((o[1].x - o[1].y) * r, (o[1].x + o[1].y) * r)
                  : make_c((o[1].x + o[1].y) * r, (o[1].y - o[1].x) * r);
  cpx<T> o2 = mul_mi<T, INV>(o[2]);
  cpx<T> o3 = INV ? make_c((-o[3].x - o[3].y) * r, (o[3].x - o[3].y) * r)
                  : make_c((o[3].y - o[3].x) * r, (-o[3].x - o[3].y) * r);
  a[0] = e[0] + o[0];
  a[4] = e[0] - o[0];
  a[1] = e[1] + o1;
  a[5] = e[1] - o1;
  a[2] = e[2] + o2;
  a[6] = e[2] - o2;
  a[3] = e[3] + o3;
  a[7] = e[3] - o3;
}

// W3 = exp(-+2 pi i/3): X1 = m + s, X2 = m - s, m = a0 - (a1+a2)/2,
// s = -+i (sqrt3/2)(a1 - a2)
template <typename T, bool INV>
__device__ __forceinline__ void dft3(cpx<T>* a) {
  const T c = kconst<T>(0x1.bb67ae8584caap-1, 0x1.cec95d0b5c1e3p-55);  // sqrt3/2
  cpx<T> t1 = a[1] + a[2], t2 = a[1] - a[2];
  cpx<T> m = make_c(a[0].x - (T)0.5 * t1.x, a[0].y - (T)0.5 * t1.y);
  cpx<T> sv = INV ? make_c(-c * t2.y, c * t2.x) : make_c(c * t2.y, -c * t2.x);
  a[0] = a[0] + t1;
  a[1] = m + sv;
  a[2] = m - sv;
}

// 6 = 2 x 3: E = DFT3(even), O = DFT3(odd), X[k] = E[k] + W6^k O[k],
// X[k+3] = E[k] - W6^k O[k]
template <typename T, bool INV>
__device__ __forceinline__ void dft6(cpx<T>* a) {
  const T c = kconst<T>(0x1.bb67ae8584caap-1, 0x1.cec95d0b5c1e3p-55);  // sqrt3/2
  cpx<T> e[3] = {a[0], a[2], a[4]};
  cpx<T> o[3] = {a[1], a[3], a[5]};
  dft3<T, INV>(e);
  dft3<T, INV>(o);
  // W6 = 1/2 -+ i sqrt3/2, W6^2 = -1/2 -+ i sqrt3/2
  const T s = INV ? c : -c;
  cpx<T> o1 = cmul(o[1], make_c((T)0.5, s));
  cpx<T> o2 = cmul(o[2], make_c((T)-0.5, s));
  a[0] = e[0] + o[0];
  a[3] = e[0] - o[0];
  a[1] = e[1] + o1;
  a[4] = e[1] - o1;
  a[2] = e[2] + o2;
  a[5] = e[2] - o2;
}

template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_small(cpx<T>* a) {
  if constexpr (R == 2) dft2<T, INV>(a);
  else if constexpr (R == 3) dft3<T, INV>(a);
  else if constexpr (R == 4) dft4<T, INV>(a);
  else if constexpr (R == 6) dft6<T, INV>(a);
  else if constexpr (R == 8) dft8<T, INV>(a);
  else static_assert(R == 2 || R == 3 || R == 4 || R == 6 || R == 8, "radix");
}

template <int N>
struct Split;
template <>
struct Split<16> { static constexpr int R1 = 4, R2 = 4; };
template <>
struct Split<32> { static constexpr int R1 = 4, R2 = 8; };
template <>
struct Split<64> { static constexpr int R1 = 8, R2 = 8; };
template <>
struct Split<24> { static constexpr int R1 = 3, R2 = 8; };
template <>
struct Split<48> { static constexpr int R1 = 6, R2 = 8; };

// frequency held at digit-reversed position p, and the position of frequency k
template <int N>
__device__ __forceinline__ int freq_of_pos(int p) {
  return p / Split<N>::R1 + Split<N>::R2 * (p % Split<N>::R1);
}
template <int N>
__device__ __forceinline__ int pos_of_freq(int k) {
  return k / Split<N>::R2 + Split<N>::R1 * (k % Split<N>::R2);
}
// signed representative of a cyclic frequency (Nyquist -> -N/2; only |k| used)
template <int N>
__device__ __forceinline__ int centred(int k) { return k < N / 2 ? k : k - N; }

// In-place length-N DFT of `npen` pencils.  Element e of pencil p is at
// base[p * ps + e * es].  PMAJOR: consecutive threads take consecutive
// pencils (good when ps == 1); otherwise consecutive threads take
// consecutive sub-transforms of one pencil (good when es == 1).
template <typename T, int N, bool INV, bool PMAJOR>
__device__ __forceinline__ void smem_fft(cpx<T>* base, int npen, int ps, int es) {
  constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
  if constexpr (!INV) {
    for (int t = threadIdx.x; t < npen * R1; t += blockDim.x) {
      int p = PMAJOR ? t % npen : t / R1;
      int n1 = PMAJOR ? t / npen : t % R1;
      cpx<T>* x = base + p * ps;
      cpx<T> v[R2];
#pragma unroll
      for (int i = 0; i < R2; ++i) v[i] = x[(n1 + R1 * i) * es];
      dft_small<T, R2, false>(v);
#pragma unroll
      for (int k = 0; k < R2; ++k) x[(n1 + R1 * k) * es] = k == 0 ? v[0] : cmul(v[k], twN<T, N>(n1 * k));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < npen * R2; t += blockDim.x) {
      int p = PMAJOR ? t % npen : t / R2;
      int k2 = PMAJOR ? t / npen : t % R2;
      cpx<T>* x = base + p * ps + R1 * k2 * es;
      cpx<T> v[R1];
#pragma unroll
      for (int i = 0; i < R1; ++i) v[i] = x[i * es];
      dft_small<T, R1, false>(v);
#pragma unroll
      for (int i = 0; i < R1; ++i) x[i * es] = v[i];
    }
    __syncthreads();
  } else {
    for (int t = threadIdx.x; t < npen * R2; t += blockDim.x) {
      int p = PMAJOR ? t % npen : t / R2;
      int k2 = PMAJOR ? t / npen : t % R2;
      cpx<T>* x = base + p * ps + R1 * k2 * es;
      cpx<T> v[R1];
#pragma unroll
      for (int i = 0; i < R1; ++i) v[i] = x[i * es];
      dft_small<T, R1, true>(v);
#pragma unroll
      for (int i = 0; i < R1; ++i) x[i * es] = v[i];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < npen * R1; t += blockDim.x) {
      int p = PMAJOR ? t % npen : t / R1;
      int n1 = PMAJOR ? t / npen : t % R1;
      cpx<T>* x = base + p * ps;
      cpx<T> v[R2];
#pragma unroll
      for (int k = 0; k < R2; ++k) {
        cpx<T> a = x[(n1 + R1 * k) * es];
        v[k] = k == 0 ? a : cmulc(a, twN<T, N>(n1 * k));
      }
      dft_small<T, R2, true>(v);
#pragma unroll
      for (int i = 0; i < R2; ++i) x[(n1 + R1 * i) * es] = v[i];
    }
    __syncthreads();
  }
}

}  // namespace lbo

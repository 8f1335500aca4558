// Register-resident 32-point transforms with compile-time twiddles.
//
// One thread holds a whole pencil of 32 complex values.  The transform is a
// radix-2 decimation in time: the bit-reversed reading of the input is a
// renaming of registers, then five stages of butterflies run in place and
// leave the output in natural order.  A butterfly whose twiddle is 1 or -+i
// takes four additions; every other one uses the scaled twiddle W = sc (1 +
// i q) (or sc (q + i)) with |q| <= 1 (twiddles_hi.h) and takes six fused
// multiply-adds: p = b (1 + i q) in two, a +- sc p in four (the scaled
// butterfly of Linzer and Feig, IBM J. Res. Dev. 37 (1993)).  A 32-point
// transform costs 388 floating-point instructions (184 additions, 204 fused
// multiply-adds; the two-stage 4 x 8 transform of fft.cuh: 448).
//
// Used where the FP64 pipe bounds the kernel (lin_reg64.cuh): on GB300 it
// issues about one warp instruction per 18 SM clocks whatever the mix, so
// the count is the cost.  The fused FP32 kernels keep their 4 x 8
// in-register transform (fused32.cuh): they are latency-bound, and the five
// dependent stages here measured slower there (1.001 against 0.965 ms for
// the gain kernel at N = 32, batch 256).
//
// Host code can include this header (tests compile it with a host compiler).
#pragma once
#include <cmath>

#include "twiddles_hi.h"

namespace lbo {
namespace reg {

template <typename T>
struct c2 {
  T x, y;
};

LBO_HD inline double fmadd(double a, double b, double c) { return fma(a, b, c); }
LBO_HD inline float fmadd(float a, float b, float c) { return fmaf(a, b, c); }

LBO_HD constexpr int brev5(int i) {
  return ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
}

// (a, b) <- (a + W b, a - W b), W = W_32^m (forward) or its conjugate (inverse)
template <typename T, bool INV, typename C>
LBO_HD inline void butterfly(C& a, C& b, int m) {
  if (m == 0) {
    const C t = a;
    a.x = t.x + b.x;
    a.y = t.y + b.y;
    b.x = t.x - b.x;
    b.y = t.y - b.y;
    return;
  }
  if (m == 8) {  // W = -i (forward), +i (inverse)
    const T vx = INV ? -b.y : b.y, vy = INV ? b.x : -b.x;
    const C t = a;
    a.x = t.x + vx;
    a.y = t.y + vy;
    b.x = t.x - vx;
    b.y = t.y - vy;
    return;
  }
  const ScaledTw w = scaled_tw32(m);
  // the conjugate: sc (1 - i q) for kind 0, -sc (-q + i) for kind 1
  const T q = (T)(INV ? -w.q : w.q);
  const T sc = (T)(INV && w.kind ? -w.sc : w.sc);
  T px, py;
  if (w.kind == 0) {  // b (1 + i q)
    px = fmadd(-q, b.y, b.x);
    py = fmadd(q, b.x, b.y);
  } else {  // b (q + i)
    px = fmadd(q, b.x, -b.y);
    py = fmadd(q, b.y, b.x);
  }
  const C t = a;
  a.x = fmadd(sc, px, t.x);
  a.y = fmadd(sc, py, t.y);
  b.x = fmadd(-sc, px, t.x);
  b.y = fmadd(-sc, py, t.y);
}

// one radix-2 stage of butterfly span HALF: 16 butterflies, each on y[b + j]
// and y[b + j + HALF], b a multiple of 2 HALF, j < HALF, twiddle W_(2 HALF)^j
template <typename T, bool INV, int HALF, typename C>
LBO_HD inline void stage32(C (&y)[32]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int j = k % HALF, b = (k / HALF) * (2 * HALF);
    butterfly<T, INV>(y[b + j], y[b + j + HALF], j * (16 / HALF));
  }
}

// x <- DFT_32(x): forward exp(-2 pi i n k / 32), inverse the conjugate
// (unnormalised).  C is any type with members x, y of type T.
template <typename T, bool INV, typename C>
LBO_HD inline void fft32(C (&x)[32]) {
  C y[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) y[i] = x[brev5(i)];
  stage32<T, INV, 1>(y);
  stage32<T, INV, 2>(y);
  stage32<T, INV, 4>(y);
  stage32<T, INV, 8>(y);
  stage32<T, INV, 16>(y);
#pragma unroll
  for (int i = 0; i < 32; ++i) x[i] = y[i];
}

}  // namespace reg
}  // namespace lbo

// Host-only check of the register-resident 32-point transform (csrc/fft_reg.cuh,
// the transform of the FP64 register kernels) and of its scaled twiddles:
// random inputs against a direct DFT summed in long double.  Prints one line
// "<type> <direction> <max relative error>" per case and "twiddle <max error>".
// Runs no kernel.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_2503_09580_gb300/csrc/fft_reg.cuh"

using namespace lbo::reg;

template <typename T, bool INV>
static double worst(int trials) {
  std::mt19937_64 rng(11);
  std::normal_distribution<double> nd;
  const long double pi = 3.141592653589793238462643383279502884L;
  double err = 0.0;
  for (int tr = 0; tr < trials; ++tr) {
    c2<T> x[32];
    long double xr[32], xi[32];
    for (int i = 0; i < 32; ++i) {
      x[i].x = (T)nd(rng);
      x[i].y = (T)nd(rng);
      xr[i] = x[i].x;
      xi[i] = x[i].y;
    }
    fft32<T, INV>(x);
    long double num = 0, den = 0;
    for (int k = 0; k < 32; ++k) {
      long double sr = 0, si = 0;
      for (int n = 0; n < 32; ++n) {
        const long double a = (INV ? 2 : -2) * pi * ((n * k) % 32) / 32;
        sr += xr[n] * cosl(a) - xi[n] * sinl(a);
        si += xr[n] * sinl(a) + xi[n] * cosl(a);
      }
      num = fmaxl(num, fmaxl(fabsl(x[k].x - sr), fabsl(x[k].y - si)));
      den = fmaxl(den, fmaxl(fabsl(sr), fabsl(si)));
    }
    err = fmax(err, (double)(num / den));
  }
  return err;
}

int main() {
  std::printf("double forward %.3e\n", worst<double, false>(200));
  std::printf("double inverse %.3e\n", worst<double, true>(200));
  std::printf("float forward %.3e\n", worst<float, false>(200));
  std::printf("float inverse %.3e\n", worst<float, true>(200));
  const long double pi = 3.141592653589793238462643383279502884L;
  double tw = 0.0;
  for (int m = 0; m < 16; ++m) {
    const ScaledTw w = scaled_tw32(m);
    const long double c = cosl(-2 * pi * m / 32), s = sinl(-2 * pi * m / 32);
    const long double wr = w.kind ? (long double)w.sc * w.q : (long double)w.sc;
    const long double wi = w.kind ? (long double)w.sc : (long double)w.sc * w.q;
    tw = fmax(tw, (double)fmaxl(fabsl(wr - c), fabsl(wi - s)));
    if (fabs(w.q) > 1.0) tw = 1.0;  // |q| <= 1 is what keeps the butterflies accurate
  }
  std::printf("twiddle %.3e\n", tw);
  return 0;
}

// Host-only check of the moment coarse correction's banded LU with an arrow
// row and column (csrc/coarse.cu): random block-tridiagonal systems with nb x
// nb blocks, with and without the rank-one border, solved and multiplied
// back.  Prints "nb nx border relative_residual" per case.  Runs no kernel.
#include <cstdio>
#include <random>

#include "../../paper_2503_09580_gb300/csrc/coarse.cu"

namespace lbo {
lbo_status solver_apply_op(lbo_solver*, const double*, double*, bool, bool) { return LBO_OK; }
void solver_axpby(lbo_solver*, double*, const double*, double, double) {}
lbo_status cuda_fail(cudaError_t, const char*) { return LBO_ECUDA; }
ProfScope::ProfScope(lbo_plan*, const char*, cudaStream_t) {}
ProfScope::~ProfScope() {}
}  // namespace lbo
using namespace lbo;

int main() {
  std::mt19937_64 rng(7);
  std::normal_distribution<double> nd;
  const int cases[][3] = {{5, 7, 0}, {5, 8, 1}, {5, 40, 1}, {13, 9, 0}, {13, 30, 1}};
  for (const auto& cs : cases) {
    const int nb = cs[0], nx = cs[1], border = cs[2];
    CoarseState C;
    C.nx = nx;
    C.nb = nb;
    C.nc = nb * nx;
    C.kl = C.ku = 2 * nb - 1;
    C.bw = 2 * C.kl + C.ku + 1;
    const int n = C.nc;
    C.ab.assign((size_t)n * C.bw, 0.0);
    C.pc.assign(n, 0.0);
    C.qr.assign(n, 0.0);
    C.d = -1.0;
    std::vector<double> D((size_t)(n + 1) * (n + 1), 0.0);  // the same system, dense
    for (int i = 0; i < nx; ++i)
      for (int j = (i > 0 ? i - 1 : 0); j <= (i < nx - 1 ? i + 1 : nx - 1); ++j)
        for (int a = 0; a < nb; ++a)
          for (int b = 0; b < nb; ++b) {
            const double v = nd(rng) + (i == j && a == b ? 3.0 : 0.0);
            at(&C, nb * i + a, nb * j + b) = v;
            D[(size_t)(nb * i + a) * (n + 1) + nb * j + b] = v;
          }
    if (border)
      for (int r = 0; r < n; ++r) {
        C.pc[r] = nd(rng);
        C.qr[r] = nd(rng);
        D[(size_t)r * (n + 1) + n] = C.pc[r];
        D[(size_t)n * (n + 1) + r] = C.qr[r];
      }
    std::vector<double> rhs(n), x(n);
    for (int r = 0; r < n; ++r) rhs[r] = x[r] = nd(rng);
    if (!factor(&C)) {
      std::printf("%d %d %d factor_failed\n", nb, nx, border);
      continue;
    }
    solve(&C, x.data());
    double s = 0;  // the border multiplier s = q^T x
    for (int r = 0; r < n; ++r) s += D[(size_t)n * (n + 1) + r] * x[r];
    double err = 0, scale = 0;
    for (int r = 0; r < n; ++r) {
      double acc = D[(size_t)r * (n + 1) + n] * s;
      for (int c = 0; c < n; ++c) acc += D[(size_t)r * (n + 1) + c] * x[c];
      err = std::max(err, std::fabs(acc - rhs[r]));
      scale = std::max(scale, std::fabs(rhs[r]));
    }
    std::printf("%d %d %d %.3e\n", nb, nx, border, err / scale);
  }
  return 0;
}

// Host-only dump of the mixed-N solver's one-axis resampling matrices
// (csrc/mixed.cu, built in long double from the trigonometric interpolant):
// for each pair "na nb" on the input, prints nb * na values row by row.
// Runs no kernel.
#include <cstdio>

#include "../../paper_2503_09580_gb300/csrc/mixed.cu"

namespace lbo {
lbo_status cuda_fail(cudaError_t, const char*) { return LBO_ECUDA; }
ProfScope::ProfScope(lbo_plan*, const char*, cudaStream_t) {}
ProfScope::~ProfScope() {}
double solver_norm2(lbo_solver*, const double*, lbo_status*) { return 0; }
void solver_axpby(lbo_solver*, double*, const double*, double, double) {}
lbo_status solver_sweep_uniform(lbo_solver*, const double*, double*, int, double) { return LBO_OK; }
}  // namespace lbo
lbo_status lbo_apply_linearized(lbo_plan*, const double*, const double*, double*, int) { return LBO_OK; }
lbo_status lbo_apply_quadratic(lbo_plan*, const double*, double*, int) { return LBO_OK; }

int main(int argc, char** argv) {
  const double L = argc > 1 ? atof(argv[1]) : 8.0;
  int na, nb;
  while (std::scanf("%d %d", &na, &nb) == 2) {
    std::vector<double> R = lbo::resample_matrix(na, nb, L);
    for (size_t i = 0; i < R.size(); ++i) std::printf("%.17e\n", R[i]);
  }
  return 0;
}

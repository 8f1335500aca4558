// Quadratic collision operator Q(f,f) in the M-point form of Eq. (2.14).
//
// With F = FFT(f), for every radial node g_j and hemisphere node sigma_m,
// alpha = pi g_j sigma_m / (2L) and the phase multiplier
// E(k) = prod_d e^{i alpha_d k_d} (cos(alpha_d N/2) at the Nyquist index,
// the average over the two images):
//   T+ = InvFFT(F E),  T- = InvFFT(F conj(E))     (both real fields)
//   T+ T- = A_c^2 - B_s^2, the real-space form of I_{j,k,m}
//   Q^+ = 16 pi^2 sum_j w_j B(g_j) s_{j,k} FFT( sum_m w_m T+ T- )
//   Q   = InvFFT(Q^+) - f InvFFT(F omega).
// The sum over m is taken in real space before the forward transform of
// each j (the transform is linear), so one application costs 2 J M inverse
// transforms + J forward transforms + 4.
#include <algorithm>
#include <cmath>
#include <vector>

#include "quad_generic.cuh"

namespace lbo {

namespace {

// Product hemisphere rule: p Gauss-Legendre nodes in cos(theta) on (0, 1)
// times 2p equispaced azimuths; weights sum to 1 (Eq. (2.13) carries 2 pi).
void hemisphere_rule(int p, std::vector<double>& sig, std::vector<double>& wm) {
  std::vector<double> x, w;
  gauss_legendre(p, x, w);
  const int na = 2 * p;
  sig.clear();
  wm.clear();
  for (int a = 0; a < p; ++a) {
    const double mu = 0.5 * (x[a] + 1.0), st = std::sqrt(1.0 - mu * mu);
    for (int b = 0; b < na; ++b) {
      const double ph = (b + 0.5) * (2.0 * 3.141592653589793238462643383279502884 / na);
      sig.push_back(st * std::cos(ph));
      sig.push_back(st * std::sin(ph));
      sig.push_back(mu);
      wm.push_back(0.5 * w[a] / na);
    }
  }
}

}  // namespace

void free_quadratic(lbo_plan* p) {
  QuadState* qs = (QuadState*)p->quad;
  if (!qs) return;
  if (qs->ws) cudaFree(qs->ws);
  if (qs->d_gsw) cudaFree(qs->d_gsw);
  delete qs;
  p->quad = nullptr;
}

lbo_status apply_quadratic_device(lbo_plan* p, const double* f, double* out, int B) {
  if (is_split16_precision(p->precision)) {
    set_error_text("Q(f,f) is not built in the split 16-bit precisions (give the solver an FP64 or FP32 "
                   "residual plan)");
    return LBO_EUNSUPPORTED;
  }
  cudaError_t e = upload_twiddles();
  if (e != cudaSuccess) return cuda_fail(e, "quadratic twiddles");
  QuadState* qs = (QuadState*)p->quad;
  if (!qs) {
    qs = new QuadState();
    p->quad = qs;
  }
  if (qs->p != p->hemi_p) {
    hemisphere_rule(p->hemi_p, qs->sig, qs->wm);
    qs->p = p->hemi_p;
  }
  const bool fused = p->precision == LBO_PREC_FP32 && p->N == 32 && p->kernel_choice == 0;
  const int G = fused ? (p->jgroups > 0 ? std::min(p->jgroups, p->J) : std::min(fused32_default_groups(B), p->J)) : 0;
  const size_t N = p->N, H = N * N * (N / 2 + 1), n3 = N * N * N;
  const int M = (int)qs->wm.size();
  const size_t rb = generic_real_bytes(p->precision);
  const size_t MB = fused ? 0 : (size_t)q_chunk(B, M, (int)N, rb);
  const size_t need = fused ? quad_fused32_workspace_bytes(B, G)
                            : (size_t)B * (4 * H * 2 * rb + 3 * n3 * rb) + MB * (size_t)B * (2 * H * 2 * rb + n3 * rb);
  if (need > qs->ws_bytes) {
    if (qs->ws) cudaFree(qs->ws);
    qs->ws = nullptr;
    qs->ws_bytes = 0;
    e = cudaMalloc(&qs->ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error_text("quadratic workspace allocation");
      return LBO_ENOMEM;
    }
    qs->ws_bytes = need;
  }
  {
    // radial nodes, hemisphere nodes and weights on the device
    if (qs->gsw_p != qs->p || qs->gsw_plan_tables != (const void*)p->d_phi32) {
      if (qs->d_gsw) cudaFree(qs->d_gsw);
      qs->d_gsw = nullptr;
      std::vector<double> h(p->gj);
      h.insert(h.end(), qs->sig.begin(), qs->sig.end());
      h.insert(h.end(), qs->wm.begin(), qs->wm.end());
      e = cudaMalloc(&qs->d_gsw, sizeof(double) * h.size());
      if (e == cudaSuccess) e = cudaMemcpy(qs->d_gsw, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "quadrature nodes upload");
      qs->gsw_p = qs->p;
      qs->gsw_plan_tables = p->d_phi32;
    }
  }
  if (fused) {
    int launches = 0;
    lbo_status st = run_quadratic_fused32(p, f, out, B, qs->ws, qs->d_gsw, (int)qs->wm.size(), G, &launches);
    if (st == LBO_OK && (p->mass_fix || p->moment_fix))
      st = launch_fixes(p, out, B, p->N, 2.0 * p->L / p->N, p->stream, &launches);
    p->last_launches = launches;
    return st;
  }
  switch (p->precision) {
    case LBO_PREC_FP64: return dispatch_q<double>(p, qs, f, out, B, p->d_phi64, p->d_omega64);
    case LBO_PREC_FP32: return dispatch_q<float>(p, qs, f, out, B, p->d_phi32, p->d_omega32);
    default: return run_quadratic_twofold(p, qs, f, out, B);
  }
}

}  // namespace lbo

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

// Loss multiplier of Eq. (2.16) per half-spectrum position (p1, p2, k3):
//   16 pi^2 / N^3 sum_j w_j B(g_j) sum_m w_m cos(pi g_j sigma_m . k / L),
// the cosine as Re prod_d E_d(k_d)^2 with E_d the gain's per-axis phase
// factor exp(i alpha_d k_d), alpha = pi g_j sigma_m / (2L), which is
// cos(alpha_d N/2) at the Nyquist index: so the squared factor is
// exp(2 i alpha_d k_d) off the Nyquist planes and cos^2(alpha_d N/2) on them,
// the gain's own kernel at k = 0, which makes Q^_0 vanish (Sec. 2.3):
// fac[(jm 3 + d) N + cyclic k], weights wjm = w_j B_j w_m.
template <int N>
__global__ void k_omega_quadrature(const double2* __restrict__ fac, const double* __restrict__ wjm, int JM,
                                   double scale, double* __restrict__ out) {
  constexpr int HC = N / 2 + 1, NC = N * HC;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * NC; t += gridDim.x * blockDim.x) {
    const int r = t / NC, col = t % NC, p2 = col / HC, k3 = col % HC;
    const int c1 = freq_of_pos<N>(r), c2 = freq_of_pos<N>(p2);
    double acc = 0.0;
    for (int jm = 0; jm < JM; ++jm) {
      const double2 a = fac[(size_t)(jm * 3 + 0) * N + c1], b = fac[(size_t)(jm * 3 + 1) * N + c2];
      const double2 c = fac[(size_t)(jm * 3 + 2) * N + k3];
      const double abr = a.x * b.x - a.y * b.y, abi = a.x * b.y + a.y * b.x;
      acc += wjm[jm] * (abr * c.x - abi * c.y);
    }
    out[t] = scale * acc;
  }
}

template <typename T>
__global__ void k_to_transform_type(const double* __restrict__ a, T* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b[i] = T(a[i]);
}

// The Eq. (2.16) multiplier in the plan's transform precision, rebuilt when
// the precision, the hemisphere rule or the tables change.
lbo_status ensure_omega_quadrature(lbo_plan* p, QuadState* qs) {
  if (qs->d_omq && qs->omq_prec == p->precision && qs->omq_p == qs->p && qs->omq_tables == (const void*)p->d_phi64)
    return LBO_OK;
  if (qs->d_omq) cudaFree(qs->d_omq);
  qs->d_omq = nullptr;
  const int N = p->N, J = p->J, M = (int)qs->wm.size();
  const size_t H = (size_t)N * N * (N / 2 + 1);
  const double pi = 3.141592653589793238462643383279502884;
  std::vector<double2> fac((size_t)J * M * 3 * N);
  std::vector<double> wjm((size_t)J * M);
  for (int j = 0; j < J; ++j)
    for (int m = 0; m < M; ++m) {
      const size_t jm = (size_t)j * M + m;
      wjm[jm] = p->wj[j] * p->Bj[j] * qs->wm[m];
      for (int d = 0; d < 3; ++d) {
        const double al = pi * p->gj[j] * qs->sig[3 * m + d] / (2.0 * p->L);  // the gain's alpha_d
        const double cn = std::cos(al * (N / 2));
        for (int k = 0; k < N; ++k) {
          const int kc = k < N / 2 ? k : k - N;
          fac[(jm * 3 + d) * N + k] = kc == -N / 2 ? make_double2(cn * cn, 0.0)
                                                   : make_double2(std::cos(2.0 * al * kc), std::sin(2.0 * al * kc));
        }
      }
    }
  double2* d_fac = nullptr;
  double *d_w = nullptr, *d_out = nullptr;
  const size_t rb = p->precision == LBO_PREC_FP32 ? 4 : generic_real_bytes(p->precision);
  cudaError_t e = cudaMalloc(&d_fac, sizeof(double2) * fac.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_w, sizeof(double) * wjm.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(double) * H);
  if (e == cudaSuccess) e = cudaMalloc(&qs->d_omq, rb * H);
  if (e == cudaSuccess) e = cudaMemcpy(d_fac, fac.data(), sizeof(double2) * fac.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_w, wjm.data(), sizeof(double) * wjm.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const double scale = 16.0 * pi * pi / ((double)N * N * N);
    const int grid = (int)std::min<size_t>((H + 255) / 256, 152 * 8);
    switch (N) {
      case 16: k_omega_quadrature<16><<<grid, 256, 0, p->stream>>>(d_fac, d_w, J * M, scale, d_out); break;
      case 24: k_omega_quadrature<24><<<grid, 256, 0, p->stream>>>(d_fac, d_w, J * M, scale, d_out); break;
      case 32: k_omega_quadrature<32><<<grid, 256, 0, p->stream>>>(d_fac, d_w, J * M, scale, d_out); break;
      case 48: k_omega_quadrature<48><<<grid, 256, 0, p->stream>>>(d_fac, d_w, J * M, scale, d_out); break;
      default: k_omega_quadrature<64><<<grid, 256, 0, p->stream>>>(d_fac, d_w, J * M, scale, d_out); break;
    }
    switch (p->precision) {
      case LBO_PREC_FP64:
        e = cudaMemcpyAsync(qs->d_omq, d_out, sizeof(double) * H, cudaMemcpyDeviceToDevice, p->stream);
        break;
      case LBO_PREC_FP32: k_to_transform_type<float><<<grid, 256, 0, p->stream>>>(d_out, (float*)qs->d_omq, H); break;
      case LBO_PREC_FP32X2: k_to_transform_type<f32x2><<<grid, 256, 0, p->stream>>>(d_out, (f32x2*)qs->d_omq, H); break;
      default: k_to_transform_type<f64x2><<<grid, 256, 0, p->stream>>>(d_out, (f64x2*)qs->d_omq, H); break;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (d_fac) cudaFree(d_fac);
  if (d_w) cudaFree(d_w);
  if (d_out) cudaFree(d_out);
  if (e != cudaSuccess) {
    if (qs->d_omq) cudaFree(qs->d_omq);
    qs->d_omq = nullptr;
    return cuda_fail(e, "Eq. (2.16) loss multiplier");
  }
  qs->omq_prec = p->precision;
  qs->omq_p = qs->p;
  qs->omq_tables = p->d_phi64;
  return LBO_OK;
}

}  // namespace

void free_quadratic(lbo_plan* p) {
  QuadState* qs = (QuadState*)p->quad;
  if (!qs) return;
  if (qs->ws) cudaFree(qs->ws);
  if (qs->d_gsw) cudaFree(qs->d_gsw);
  if (qs->d_omq) cudaFree(qs->d_omq);
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
  // the fused FP32 kernels take the radial loss multiplier only
  const bool fused = p->precision == LBO_PREC_FP32 && p->N == 32 && p->kernel_choice == 0 && !p->q_sinc_quad;
  const int G = fused ? (p->jgroups > 0 ? std::min(p->jgroups, p->J) : std::min(fused32_default_groups(B), p->J)) : 0;
  const size_t N = p->N, H = N * N * (N / 2 + 1), n3 = N * N * N;
  const int M = (int)qs->wm.size();
  const size_t rb = generic_real_bytes(p->precision);
  const size_t MB = fused ? 0 : (size_t)q_chunk(B, M, (int)N, rb);
  // FP64 at N = 32 (register kernels): the phase-factor table after the chunk buffers
  const size_t ptab = p->precision == LBO_PREC_FP64 && N == 32 && p->kernel_choice != 2
                          ? (size_t)p->J * M * 3 * N * 2 * sizeof(double) : 0;
  const size_t need = fused ? quad_fused32_workspace_bytes(B, G)
                            : (size_t)B * (4 * H * 2 * rb + 3 * n3 * rb) + MB * (size_t)B * (2 * H * 2 * rb + n3 * rb) + ptab;
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
  const void* omq = nullptr;
  if (p->q_sinc_quad) {
    lbo_status st = ensure_omega_quadrature(p, qs);
    if (st != LBO_OK) return st;
    omq = qs->d_omq;
  }
  switch (p->precision) {
    case LBO_PREC_FP64: return dispatch_q<double>(p, qs, f, out, B, p->d_phi64, p->d_omega64, omq);
    case LBO_PREC_FP32: return dispatch_q<float>(p, qs, f, out, B, p->d_phi32, p->d_omega32, omq);
    default: return run_quadratic_twofold(p, qs, f, out, B, omq);
  }
}

}  // namespace lbo

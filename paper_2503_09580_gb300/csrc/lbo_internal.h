// Internal plan structure of liblbo (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lbo.h"

struct lbo_plan {
  int N = 0, J = 0, device = 0;
  double L = 0, omega = 0, R = 0, C = 0, eps = 1e-9;
  int cutoff = 1, mass_fix = 0, moment_fix = 0, hemi_p = 4, precision = 0;
  int kernel_choice = 0, jgroups = 0;
  int r64_planes = 0;  // planes per CTA of the FP64 register plane kernel (0: 4)
  int q_sinc_quad = 0;  // Q's loss multiplier: 1 = the hemisphere quadrature of Eq. (2.16)
  cudaStream_t stream = nullptr;
  bool tables_dirty = false;
  // radial rule (host copy)
  std::vector<double> gj, wj, Bj;
  // device tables of Algorithm 1
  double* d_phi64 = nullptr;    // [J][QMAX] phi_j(|k|^2) / N^3
  double* d_omega64 = nullptr;  // [QMAX] omega(|k|^2) / N^3
  double* d_phit64 = nullptr;   // [J][N^3] phit_j, cyclic order
  float* d_phi32 = nullptr;
  float* d_omega32 = nullptr;
  float* d_phit32 = nullptr;
  double* d_dct64 = nullptr;    // [N/2+1][N/4] DCT-I coefficients of u^_j (lin_kernels.cuh)
  float* d_dct32 = nullptr;
  double* d_dummy_params = nullptr;
  // two-fold tables {phit, phi, omega, dct}, built on first use (lin_twofold.cu)
  void* d_x2f[4] = {nullptr, nullptr, nullptr, nullptr};  // pairs of FP32
  void* d_x2d[4] = {nullptr, nullptr, nullptr, nullptr};  // pairs of FP64
  // split 16-bit tensor-core path (lin_dftmm.cu): DFT matrices {forward,
  // inverse} per operand type, the MMA-wait error flag, per-call scratch for
  // u^_j and w when the Maxwellian cache does not hold them
  void* d_wbf[2] = {nullptr, nullptr};
  void* d_wfp[2] = {nullptr, nullptr};
  void* d_tc_err = nullptr;
  void* tc_scratch = nullptr;
  size_t tc_scratch_bytes = 0;
  // reductions of the slab-block primitives (slab_block.cu)
  double* blk_red = nullptr;
  size_t blk_red_cap = 0;
  // cache of the Maxwellian-dependent factors (lbo_plan_cache_maxwellians):
  // valid for apply calls with this params pointer, batch, precision and path
  const double* mc_params = nullptr;
  int mc_batch = 0, mc_precision = -1, mc_path = -1;
  bool mc_valid = false;
  void *mc_uh = nullptr, *mc_w = nullptr;
  size_t mc_uh_bytes = 0, mc_w_bytes = 0;
  // workspace of the generic path
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // staging for host-pointer calls
  double *stage_in = nullptr, *stage_out = nullptr, *stage_par = nullptr;
  size_t stage_in_cap = 0, stage_out_cap = 0, stage_par_cap = 0;
  // quadratic operator state (hemisphere rule, workspace)
  void* quad = nullptr;
  int last_launches = 0;
  // per-kernel event timing
  bool profiling = false;
  struct ProfEvent {
    const char* name;
    cudaEvent_t start, stop;
  };
  std::vector<ProfEvent> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  struct ProfTotal {
    const char* name;
    int launches;
    double ms;
  };
  std::vector<ProfTotal> prof_totals;
};

struct lbo_solver {
  lbo_problem pb;
  lbo_plan* plan = nullptr;
  lbo_plan* rplan = nullptr;  // Q of the residual, if not the solver's own plan
  int N = 0, nx = 0, m = 0;
  size_t n3 = 0, len = 0;
  double h = 0, dx = 1, wnorm = 1, kL = 0, kR = 0;
  double *V = nullptr, *Z = nullptr;  // Krylov basis (m+1) and preconditioned vectors (m)
  double *w = nullptr, *Lv = nullptr, *rhs = nullptr, *x = nullptr, *evec = nullptr, *Qf = nullptr;
  double *params = nullptr, *nu = nullptr, *WL = nullptr, *WR = nullptr;
  double *part = nullptr, *res = nullptr;  // reduction partials, small results
  double* host = nullptr;                  // pinned small results
  void* netstate = nullptr;                // learned preconditioner (network.cu)
  void* coarse = nullptr;                  // moment coarse correction (coarse.cu)
  void* mixed = nullptr;                   // cells of different N (mixed.cu)
  bool force_sweep = false;                // fallback from the learned preconditioner
  double shift = 0, r_first = 0;           // pseudo-transient shift 1/dtau, first residual norm
  const double* fcur = nullptr;            // state of the current step (exact Jacobian)
  double fnorm = 0;                        // its Euclidean norm
  double *ja = nullptr, *jb = nullptr;     // f +- s v and their Q (exact Jacobian)
  void* devk = nullptr;                    // device-resident Arnoldi state (solver.cu)
};

namespace lbo {
lbo_status cuda_fail(cudaError_t e, const char* where);
// learned preconditioner (network.cu)
lbo_status network_correction(lbo_solver* S, const double* v, double* z);
lbo_status network_record(lbo_solver* S, const double* w, const double* zk, double* s_scratch,
                          lbo_status (*sweep)(lbo_solver*, const double*, double*));
void free_network(lbo_solver* S);
bool network_collecting(const lbo_solver* S);
// slab operator A' (with or without the mass border) and y = a x + b y (solver.cu)
lbo_status solver_apply_op(lbo_solver* S, const double* v, double* out, bool border, bool collisions);
void solver_axpby(lbo_solver* S, double* y, const double* x, double a, double b);
double solver_norm2(lbo_solver* S, const double* y, lbo_status* st);
lbo_status solver_sweep_uniform(lbo_solver* S, const double* r, double* z, int N, double h);
// cells of different N (mixed.cu)
lbo_status mixed_setup(lbo_solver* S, lbo_plan* const* plans, int nplans, const int* cell_plan);
size_t mixed_state_length(const lbo_plan* const* plans, int nx, const int* cell_plan);
void mixed_moments(lbo_solver* S, const double* f, double* params, double* nu);
lbo_status mixed_residual(lbo_solver* S, const double* f, double* out, double* nrm);
lbo_status mixed_apply_op(lbo_solver* S, const double* v, double* out);
lbo_status mixed_sweep(lbo_solver* S, const double* v, double* z);
lbo_status mixed_set_residual_plan(lbo_solver* S, lbo_plan* plan);
void free_mixed(lbo_solver* S);
// moment coarse correction (coarse.cu)
lbo_status coarse_assemble(lbo_solver* S, bool border);
bool coarse_valid(const lbo_solver* S);
lbo_status coarse_correct(lbo_solver* S, const double* v, double* z);
void free_coarse(lbo_solver* S);
void set_error_text(const char* msg);
// zero-mode removal and/or FP64 conservation projection of out[B][N^3]
lbo_status launch_fixes(lbo_plan* p, double* out, int B, int N, double h, cudaStream_t s, int* launches);
void free_quadratic(lbo_plan* p);
void gauss_legendre(int J, std::vector<double>& x, std::vector<double>& w);
lbo_status apply_quadratic_device(lbo_plan* p, const double* f, double* out, int B);
// two-fold precisions FP32X2 / FP64X2 (lin_twofold.cu)
lbo_status run_linearized_twofold(lbo_plan* p, const double* params, const double* g, double* out, int B,
                                  const void* cache_uh = nullptr, const void* cache_w = nullptr);
lbo_status precompute_twofold(lbo_plan* p, const double* params, int B, void* uh, void* w);
lbo_status twofold_tables(lbo_plan* p, const void** phi, const void** omega, const void** phit, const void** dct);
void free_twofold_tables(lbo_plan* p);
inline bool is_twofold_precision(int prec) { return prec == LBO_PREC_FP32X2 || prec == LBO_PREC_FP64X2; }
// bytes of one real number in the transform precision of the generic path
inline size_t generic_real_bytes(int prec) { return prec == LBO_PREC_FP64X2 ? 16 : 8; }
// split 16-bit precisions on the tensor cores (lin_dftmm.cu)
inline bool is_split16_precision(int prec) { return prec == LBO_PREC_BF16_SPLIT || prec == LBO_PREC_FP16_SPLIT; }
bool dftmm_supported(int N);
lbo_status run_linearized_dftmm(lbo_plan* p, const double* params, const double* g, double* out, int B,
                                const float* uh, const float* w, void* ws);
lbo_status dftmm_check(lbo_plan* p);
void free_dftmm(lbo_plan* p);
// fused FP32 path for N = 32 (lin_fused32.cu)
size_t fused32_workspace_bytes(int B, int G, int J);
int fused32_default_groups(int B);
lbo_status run_linearized_fused32(lbo_plan* p, const double* params, const double* g, double* out, int B,
                                  void* ws, int G, int* launches, const float* cached_uhat = nullptr);
size_t fused32_uhat_bytes(int B, int J);
lbo_status precompute_fused32(lbo_plan* p, const double* params, int B, float* uhat);
size_t quad_fused32_workspace_bytes(int B, int G);
lbo_status run_quadratic_fused32(lbo_plan* p, const double* f, double* out, int B, void* ws, const double* d_gsw,
                                 int M, int G, int* launches);
void free_profile(lbo_plan* p);

// Raises a kernel's dynamic shared-memory limit to `bytes` once per device
// (the 48 KB default bounds dynamic and static shared memory together): the
// attribute stays with the function, so later launches -- including those
// recorded into a CUDA graph -- do not set it again.
void raise_smem_limit(const void* func, size_t bytes);

// Event bracket around one launch when profiling is on.
struct ProfScope {
  lbo_plan* p;
  const char* name;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(lbo_plan* plan, const char* n, cudaStream_t s);
  ~ProfScope();
  cudaStream_t s;
};
}  // namespace lbo

// Launch a kernel on stream s of plan p under a profiling scope.
#define LBO_LAUNCH(p, name, s, kernel, grid, block, smem, ...)      \
  do {                                                              \
    lbo::ProfScope _ps((p), (name), (s));                           \
    kernel<<<(grid), (block), (smem), (s)>>>(__VA_ARGS__);          \
  } while (0)

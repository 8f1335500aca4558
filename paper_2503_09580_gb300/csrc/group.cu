// Groups of plans applied together (mixed grid sizes in one launch
// sequence), CUDA-graph replay, and the launch-shape autotuner.
#include <cstring>
#include <vector>

#include "lbo_internal.h"

struct lbo_group {
  std::vector<lbo_plan*> plans;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  cudaStream_t stream = nullptr;  // the caller's stream
  bool use_graph = false;
  // cached graph and the call signature it was recorded with
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> sig;
  int calls_with_sig = 0;
};

namespace {

lbo_status run_members(lbo_group* G, const double* const* params, const double* const* g, double* const* out,
                       const int* batch) {
  cudaError_t e = cudaEventRecord(G->fork, G->stream);
  if (e != cudaSuccess) return lbo::cuda_fail(e, "group fork");
  lbo_status st = LBO_OK;
  for (size_t i = 0; i < G->plans.size() && st == LBO_OK; ++i) {
    lbo_plan* p = G->plans[i];
    cudaStream_t keep = p->stream;
    e = cudaStreamWaitEvent(G->streams[i], G->fork, 0);
    if (e != cudaSuccess) return lbo::cuda_fail(e, "group wait");
    p->stream = G->streams[i];
    st = lbo_apply_linearized(p, params[i], g[i], out[i], batch[i]);
    p->stream = keep;
    if (st == LBO_OK) {
      e = cudaEventRecord(G->done[i], G->streams[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(G->stream, G->done[i], 0);
      if (e != cudaSuccess) return lbo::cuda_fail(e, "group join");
    }
  }
  return st;
}

}  // namespace

extern "C" {

lbo_status lbo_group_create(lbo_plan* const* plans, int nplans, lbo_group** out) {
  if (!plans || nplans < 1 || nplans > 64 || !out) return LBO_EINVAL;
  *out = nullptr;
  for (int i = 0; i < nplans; ++i)
    if (!plans[i]) return LBO_EINVAL;
  lbo_group* G = new lbo_group();
  cudaError_t e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming);
  for (int i = 0; i < nplans && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    G->plans.push_back(plans[i]);
    G->streams.push_back(s);
    G->done.push_back(ev);
  }
  if (e != cudaSuccess) {
    lbo_group_destroy(G);
    return lbo::cuda_fail(e, "group create");
  }
  *out = G;
  return LBO_OK;
}

lbo_status lbo_group_set_stream(lbo_group* G, void* stream) {
  if (!G) return LBO_EINVAL;
  G->stream = (cudaStream_t)stream;
  return LBO_OK;
}

lbo_status lbo_group_use_graph(lbo_group* G, int enable) {
  if (!G) return LBO_EINVAL;
  G->use_graph = enable != 0;
  return LBO_OK;
}

lbo_status lbo_group_apply_linearized(lbo_group* G, const double* const* params, const double* const* g,
                                      double* const* out, const int* batch) {
  if (!G || !params || !g || !out || !batch) return LBO_EINVAL;
  const size_t n = G->plans.size();
  if (!G->use_graph) return run_members(G, params, g, out, batch);
  std::vector<const void*> sig;
  for (size_t i = 0; i < n; ++i) {
    sig.push_back(params[i]);
    sig.push_back(g[i]);
    sig.push_back(out[i]);
    sig.push_back((const void*)(size_t)batch[i]);
  }
  if (G->exec && sig == G->sig) {
    cudaError_t e = cudaGraphLaunch(G->exec, G->stream);
    return e == cudaSuccess ? LBO_OK : lbo::cuda_fail(e, "graph launch");
  }
  if (sig != G->sig) {
    G->sig = sig;
    G->calls_with_sig = 0;
    if (G->exec) {
      cudaGraphExecDestroy(G->exec);
      G->exec = nullptr;
    }
  }
  // the first call with a new signature runs eagerly (tables, workspaces and
  // one-time uploads happen outside any capture); the second records it
  if (G->calls_with_sig++ == 0 || G->stream == nullptr) return run_members(G, params, g, out, batch);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(G->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return lbo::cuda_fail(e, "begin capture");
  lbo_status st = run_members(G, params, g, out, batch);
  e = cudaStreamEndCapture(G->stream, &graph);
  if (st != LBO_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return lbo::cuda_fail(e, "graph instantiate");
  e = cudaGraphLaunch(G->exec, G->stream);
  return e == cudaSuccess ? LBO_OK : lbo::cuda_fail(e, "graph launch");
}

void lbo_group_destroy(lbo_group* G) {
  if (!G) return;
  if (G->exec) cudaGraphExecDestroy(G->exec);
  for (auto s : G->streams)
    if (s) cudaStreamDestroy(s);
  for (auto ev : G->done)
    if (ev) cudaEventDestroy(ev);
  if (G->fork) cudaEventDestroy(G->fork);
  delete G;
}

// Planes per CTA of the FP64 register plane kernel (N = 32): 2, 4 or 8,
// each timed over three applications after one untimed.
static lbo_status autotune_planes(lbo_plan* p, const double* params, const double* g, double* out, int batch,
                                  int* choice) {
  const int cands[] = {2, 4, 8};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  int best_p = 0;
  const int keep = p->r64_planes;
  lbo_status st = LBO_OK;
  for (int P : cands) {
    p->r64_planes = P;
    st = lbo_apply_linearized(p, params, g, out, batch);
    if (st != LBO_OK) break;
    cudaEventRecord(a, p->stream);
    for (int r = 0; r < 3 && st == LBO_OK; ++r) st = lbo_apply_linearized(p, params, g, out, batch);
    cudaEventRecord(b, p->stream);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (st == LBO_OK && ms < best) {
      best = ms;
      best_p = P;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->r64_planes = st == LBO_OK ? best_p : keep;
  if (choice) *choice = p->r64_planes;
  return st;
}

lbo_status lbo_plan_autotune(lbo_plan* p, const double* params, const double* g, double* out, int batch,
                             int* choice) {
  if (!p || batch < 1 || !params || !g || !out) return LBO_EINVAL;
  if (choice) *choice = 0;
  if (p->precision == LBO_PREC_FP64 && p->N == 32 && p->kernel_choice != 2) return autotune_planes(p, params, g, out,
                                                                                                     batch, choice);
  if (!(p->precision == LBO_PREC_FP32 && p->N == 32 && p->kernel_choice == 0)) return LBO_OK;
  const int cands[] = {1, 2, 3, 4, 6, 8};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  int best_g = 0;
  const int keep = p->jgroups;
  lbo_status st = LBO_OK;
  for (int G : cands) {
    if (G > p->J) continue;
    p->jgroups = G;
    st = lbo_apply_linearized(p, params, g, out, batch);
    if (st != LBO_OK) break;
    cudaEventRecord(a, p->stream);
    for (int r = 0; r < 3 && st == LBO_OK; ++r) st = lbo_apply_linearized(p, params, g, out, batch);
    cudaEventRecord(b, p->stream);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (st == LBO_OK && ms < best) {
      best = ms;
      best_g = G;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  p->jgroups = st == LBO_OK ? best_g : keep;
  if (choice) *choice = p->jgroups;
  return st;
}

}  // extern "C"

// Per-kernel CUDA-event timing of a plan (lbo_plan_profile*).
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "lbo_internal.h"

namespace lbo {

void raise_smem_limit(const void* func, size_t bytes) {
  // set for any size: the 48 KB default covers dynamic and static shared
  // memory together, so a request just at 48 KB still needs it
  if (bytes == 0) return;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[{func, dev}];
  if (have >= bytes) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess) have = bytes;
  else cudaGetLastError();
}

static cudaEvent_t take_event(lbo_plan* p) {
  if (!p->prof_pool.empty()) {
    cudaEvent_t e = p->prof_pool.back();
    p->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

ProfScope::ProfScope(lbo_plan* plan, const char* n, cudaStream_t st) : p(plan), name(n), s(st) {
  if (!p || !p->profiling) return;
  a = take_event(p);
  b = take_event(p);
  if (a) cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
  if (!a || !b) return;
  cudaEventRecord(b, s);
  p->prof_pending.push_back({name, a, b});
}

static void fold(lbo_plan* p) {
  if (p->prof_pending.empty()) return;
  cudaStreamSynchronize(p->stream);
  for (auto& ev : p->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.start, ev.stop) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    bool found = false;
    for (auto& t : p->prof_totals)
      if (std::strcmp(t.name, ev.name) == 0) {
        t.launches += 1;
        t.ms += ms;
        found = true;
        break;
      }
    if (!found) p->prof_totals.push_back({ev.name, 1, (double)ms});
    p->prof_pool.push_back(ev.start);
    p->prof_pool.push_back(ev.stop);
  }
  p->prof_pending.clear();
}

void free_profile(lbo_plan* p) {
  if (!p->prof_pending.empty()) cudaStreamSynchronize(p->stream);
  for (auto& ev : p->prof_pending) {
    cudaEventDestroy(ev.start);
    cudaEventDestroy(ev.stop);
  }
  for (auto e : p->prof_pool) cudaEventDestroy(e);
  p->prof_pending.clear();
  p->prof_pool.clear();
}

}  // namespace lbo

extern "C" {

lbo_status lbo_plan_profile(lbo_plan* p, int enable) {
  if (!p) return LBO_EINVAL;
  if (enable) {
    lbo::fold(p);
    p->prof_totals.clear();
  }
  p->profiling = enable != 0;
  return LBO_OK;
}

int lbo_plan_profile_count(lbo_plan* p) {
  if (!p) return 0;
  lbo::fold(p);
  return (int)p->prof_totals.size();
}

lbo_status lbo_plan_profile_get(lbo_plan* p, int i, const char** name, int* launches, double* total_ms) {
  if (!p || i < 0 || i >= (int)p->prof_totals.size()) return LBO_EINVAL;
  if (name) *name = p->prof_totals[i].name;
  if (launches) *launches = p->prof_totals[i].launches;
  if (total_ms) *total_ms = p->prof_totals[i].ms;
  return LBO_OK;
}

}  // extern "C"

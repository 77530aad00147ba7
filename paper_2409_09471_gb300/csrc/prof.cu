// Launch timing for the roofline report (see prof.cuh).
#include "prof.cuh"
#include <atomic>
#include <mutex>

namespace ttsg {

namespace {
struct Rec {
  int cls;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::mutex g_mu;
std::atomic<int> g_mask{0};  // read by every launch wrapper, without the lock
std::vector<Rec> g_recs;
}  // namespace

std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool prof_on(int cls) { return !g_dry_run && (g_mask.load(std::memory_order_relaxed) >> cls) & 1; }

int prof_begin(int cls, cudaStream_t st) {
  if (!prof_on(cls)) return -1;
  Rec r{cls, nullptr, nullptr, 0, 0};
  TT_CUDA(cudaEventCreate(&r.a));
  TT_CUDA(cudaEventCreate(&r.b));
  TT_CUDA(cudaEventRecord(r.a, st));
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end(int token, cudaStream_t st, double flops, double bytes) {
  if (token < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec& r = g_recs[token];
  r.flops = flops;
  r.bytes = bytes;
  TT_CUDA(cudaEventRecord(r.b, st));
}

}  // namespace ttsg

using namespace ttsg;

int tt_profile(int mask) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_recs.clear();
  g_mask.store(mask);
  return TT_OK;
}

int tt_profile_read(int cls, double* ms_total, int64_t* launches, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  double ms = 0, fl = 0, by = 0;
  int64_t nl = 0;
  for (auto& r : g_recs) {
    if (r.cls != cls) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return TT_ERR_CUDA;
    float t = 0;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return TT_ERR_CUDA;
    ms += t;
    fl += r.flops;
    by += r.bytes;
    ++nl;
  }
  if (ms_total) *ms_total = ms;
  if (launches) *launches = nl;
  if (flops) *flops = fl;
  if (bytes) *bytes = by;
  return TT_OK;
}

int64_t tt_launch_count(void) { return (int64_t)g_launches.load(); }

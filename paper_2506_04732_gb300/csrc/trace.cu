// Launch counter and event-based per-family kernel timing (t2s2_trace_*).
#include <atomic>
#include <mutex>
#include <vector>

#include "trace.h"

namespace t2s2 {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_on{0};
std::mutex g_mu;
struct Rec {
  int fam;
  cudaEvent_t a, b;
  double flops, bytes;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
double g_ms[kTrFamilies], g_fl[kTrFamilies], g_by[kTrFamilies];
long long g_cnt[kTrFamilies];

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
void drain_locked() {
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      g_ms[r.fam] += ms;
      g_fl[r.fam] += r.flops;
      g_by[r.fam] += r.bytes;
      g_cnt[r.fam] += 1;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}
}  // namespace

TraceScope::TraceScope(int f, cudaStream_t s, double fl, double by) : fam(f), st(s), flops(fl), bytes(by), slot(-1) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  // no timing events inside a stream capture (they would become graph nodes)
  if (g_on.load(std::memory_order_relaxed) && cudaStreamIsCapturing(st, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_recs.size() > 200000) drain_locked();
    Rec r{fam, get_event(), get_event(), flops, bytes};
    cudaEventRecord(r.a, st);
    g_recs.push_back(r);
    slot = (int)g_recs.size() - 1;
  }
}
TraceScope::~TraceScope() {
  if (slot >= 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (slot < (int)g_recs.size()) cudaEventRecord(g_recs[slot].b, st);
  }
}

void trace_add_work(int fam, double flops, double bytes) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_fl[fam] += flops;
  g_by[fam] += bytes;
}

}  // namespace t2s2

namespace t2s2 {
namespace {
// An empty kernel launched the way the library's kernels are, to measure what
// a traced launch costs beyond its work.
__global__ void k_trace_empty() {
  pdl_wait();
  pdl_trigger();
}
}  // namespace
}  // namespace t2s2

using namespace t2s2;

extern "C" {

long long t2s2_kernel_launches(void) { return g_launches.load(); }

t2s2_status t2s2_trace_overhead(int n, void* stream, double* ms) {
  if (n < 1 || !ms) return T2S2_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t a = nullptr, b = nullptr;
  T2S2_CUDA_TRY(cudaEventCreate(&a));
  T2S2_CUDA_TRY(cudaEventCreate(&b));
  double tot = 0.0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n + 1 && e == cudaSuccess; ++i) {
    e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch_pdl(k_trace_empty, 1, 32, 0, st);
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float f = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, a, b);
    if (i > 0) tot += f;  // the first launch warms up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) {
    set_last_cuda_error(e, "t2s2_trace_overhead", __FILE__, __LINE__);
    return T2S2_ECUDA;
  }
  *ms = tot / n;
  return T2S2_OK;
}

t2s2_status t2s2_trace(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  for (int f = 0; f < kTrFamilies; ++f) g_ms[f] = g_fl[f] = g_by[f] = 0.0, g_cnt[f] = 0;
  g_on.store(enable ? 1 : 0);
  return T2S2_OK;
}

t2s2_status t2s2_trace_read(int family, long long* launches, double* ms, double* flops, double* bytes) {
  if (family < 0 || family >= kTrFamilies) return T2S2_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  drain_locked();
  if (launches) *launches = g_cnt[family];
  if (ms) *ms = g_ms[family];
  if (flops) *flops = g_fl[family];
  if (bytes) *bytes = g_by[family];
  return T2S2_OK;
}
}

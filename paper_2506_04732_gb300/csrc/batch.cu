// Grouped TT apply over many independent instances in one persistent launch
// (t2s2_apply_batched), with a small autotuner for the launch shape.
//
// Every core of every instance becomes one work descriptor (ApplyCore); the
// descriptors and the prefix sums of their tile counts go to the device in
// one copy, and a persistent grid of CTAs loops over all tiles of all cores
// (apply.cu for FP64, apply_tc.cu for the tensor-core path), so instances of
// uneven n and ranks share one launch with no per-instance launch overhead.
//
// Autotuner: the tensor-core kernel comes in two variants, direct loads of
// the operand rows or staged ones (a bulk TMA copy of the next tile's rows
// into shared memory while the current tile runs, fewer CTAs per SM), and the
// persistent grid is k CTAs per SM, k up to the variant's residency limit.
// The first call with a new shape class (precision, largest m in steps of 16,
// largest rank, tile count and stage size as powers of two) times every
// (variant, k) with CUDA events (one warm-up launch, then two timed) and
// keeps the fastest in a table that later calls reuse; t2s2_autotune_report
// prints the table.  Re-running the product is harmless: it overwrites y
// with the same values.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "api_internal.h"
#include "trace.h"

namespace t2s2 {

namespace {

struct TuneKey {
  int prec, mb, rb, tb;
  long sb;
  bool operator<(const TuneKey& o) const {
    return std::tie(prec, mb, rb, tb, sb) < std::tie(o.prec, o.mb, o.rb, o.tb, o.sb);
  }
};
struct TuneVal {
  int ctas_per_sm;
  bool staged;  // the bulk-TMA staged variant of the tensor-core kernel
  std::vector<std::tuple<bool, int, float>> trials;  // (staged, ctas per SM, ms per launch)
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_table;
// grow-only staging: pinned host and device copies of the work list
char* g_host = nullptr;
char* g_dev = nullptr;
size_t g_cap = 0;
int* g_err = nullptr;

int pow2_ceil(long v) {
  int p = 1;
  while (p < v && p < (1 << 30)) p <<= 1;
  return p;
}

t2s2_status ensure_staging(size_t bytes) {
  if (bytes <= g_cap) return T2S2_OK;
  if (g_host) cudaFreeHost(g_host), g_host = nullptr;
  if (g_dev) cudaFree(g_dev), g_dev = nullptr;
  g_cap = 0;
  const size_t want = std::max(bytes, (size_t)64 << 10);
  T2S2_CUDA_TRY(cudaMallocHost(&g_host, want));
  T2S2_CUDA_TRY(cudaMalloc(&g_dev, want));
  g_cap = want;
  if (!g_err) T2S2_CUDA_TRY(cudaMalloc(&g_err, sizeof(int)));
  return T2S2_OK;
}

}  // namespace
}  // namespace t2s2

using namespace t2s2;

extern "C" {

t2s2_status t2s2_apply_batched(const t2s2_op* ops, const t2s2_tt* x, t2s2_tt* y, int count, double c_mass,
                               double c_op, t2s2_precision prec, void* stream) {
  if (!ops || !x || !y || count < 0) return T2S2_EINVAL;
  if (prec < T2S2_FP64 || prec > T2S2_BF16_REFINE) return T2S2_EINVAL;
  if (count == 0) return T2S2_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<ApplyCore> cores;
  std::vector<DevTT> ys(count);
  int mmax = 1, rmax = 1;
  for (int i = 0; i < count; ++i) {
    if (!ops[i]) return T2S2_EINVAL;
    T2S2_TRY(check_tt(ops[i], &x[i]));
    if (x[i].loc != T2S2_DEVICE || y[i].loc != T2S2_DEVICE) return T2S2_EINVAL;
    if (!y[i].r || !y[i].cores || !y[i].cap || y[i].d != ops[i]->d) return T2S2_EINVAL;
    DevTT dx;
    dx.d = x[i].d;
    for (int k = 0; k <= dx.d; ++k) dx.r[k] = x[i].r[k];
    for (int k = 0; k < dx.d; ++k) {
      dx.m[k] = x[i].m[k];
      dx.c[k] = static_cast<double*>(x[i].cores[k]);
      dx.cap[k] = x[i].cap[k];
      if (y[i].cores[k] == x[i].cores[k]) return T2S2_EINVAL;
    }
    DevTT& dy = ys[i];
    dy.d = dx.d;
    for (int k = 0; k < dx.d; ++k) {
      dy.m[k] = dx.m[k];
      dy.c[k] = static_cast<double*>(y[i].cores[k]);
      dy.cap[k] = y[i].cap[k];
    }
    ApplyBatch b;
    T2S2_TRY(apply_batch(ops[i], dx, dy, c_mass, c_op, false, b));
    for (int k = 0; k < b.ncores; ++k) {
      cores.push_back(b.c[k]);
      mmax = std::max(mmax, b.c[k].m);
      rmax = std::max(rmax, std::max(b.c[k].ra, b.c[k].rb));
    }
  }
  const int n = (int)cores.size();
  bool tc = (prec == T2S2_BF16_REFINE || prec == T2S2_TF32_REFINE) && mmax <= 64;
  // the stage the staged variant would need (-1: some core is not aligned)
  long stage = tc ? 0 : -1;
  for (int i = 0; i < n && stage >= 0; ++i) {
    const long e = apply_tc_stage_elems(cores[i]);
    stage = e < 0 ? -1 : std::max(stage, e);
  }
  if (stage > 0 && apply_tc_max_ctas_per_sm(prec, stage) < 1) stage = -1;
  std::vector<int> start(n + 1);
  double fl = 0.0, by = 0.0;
  int total = 0;
  for (int i = 0; i < n; ++i) {
    start[i] = total;
    total += tc ? apply_tc_tiles(cores[i]) : apply_fp64_tiles(cores[i]);
    apply_work_totals(cores[i], &fl, &by);
  }
  start[n] = total;
  std::lock_guard<std::mutex> lk(g_mu);
  const size_t cbytes = ((sizeof(ApplyCore) * n + 255) / 256) * 256;
  T2S2_TRY(ensure_staging(cbytes + sizeof(int) * (n + 1)));
  std::memcpy(g_host, cores.data(), sizeof(ApplyCore) * n);
  std::memcpy(g_host + cbytes, start.data(), sizeof(int) * (n + 1));
  T2S2_CUDA_TRY(cudaMemcpyAsync(g_dev, g_host, cbytes + sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
  const ApplyCore* dcores = reinterpret_cast<const ApplyCore*>(g_dev);
  const int* dstart = reinterpret_cast<const int*>(g_dev + cbytes);
  if (tc) T2S2_CUDA_TRY(cudaMemsetAsync(g_err, 0, sizeof(int), st));
  auto launch = [&](bool staged, int per_sm) -> t2s2_status {
    const int grid = std::max(1, per_sm * kNumSMs);
    if (tc) return apply_tc_grouped(dcores, dstart, n, total, grid, fl, by, prec, g_err, staged ? stage : 0, st);
    return apply_fp64_grouped(dcores, dstart, n, total, grid, fl, by, st);
  };
  // shape class: precision, largest m (steps of 16), largest rank and tile
  // count (powers of two), and the stage size (powers of two; -1: none)
  const TuneKey key{tc ? (int)prec : 0, (mmax + 15) / 16, pow2_ceil(rmax), pow2_ceil(total),
                    stage > 0 ? pow2_ceil(stage) : -1};
  // T2S2_APPLY_VARIANT=direct|staged forces one variant at its residency
  // limit, without tuning (for tests of each variant)
  const char* force = std::getenv("T2S2_APPLY_VARIANT");
  if (tc && force && (std::strcmp(force, "direct") == 0 || std::strcmp(force, "staged") == 0)) {
    const bool staged = std::strcmp(force, "staged") == 0;
    if (staged && stage <= 0) return T2S2_EINVAL;
    T2S2_TRY(launch(staged, apply_tc_max_ctas_per_sm(prec, staged ? stage : 0)));
    int herr = 0;
    T2S2_CUDA_TRY(cudaMemcpyAsync(&herr, g_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    T2S2_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < count; ++i)
      for (int k = 0; k <= ys[i].d; ++k) y[i].r[k] = ys[i].r[k];
    return herr ? T2S2_ETIMEOUT : T2S2_OK;
  }
  auto it = g_table.find(key);
  if (it == g_table.end()) {
    // tune: both variants, each up to its residency limit
    TuneVal tv{1, false, {}};
    float best = 1e30f;
    cudaEvent_t e0, e1;
    T2S2_CUDA_TRY(cudaEventCreate(&e0));
    T2S2_CUDA_TRY(cudaEventCreate(&e1));
    for (int variant = 0; variant < 2; ++variant) {
      const bool staged = variant == 1;
      if (staged && !(tc && stage > 0)) continue;
      const int kmax = tc ? apply_tc_max_ctas_per_sm(prec, staged ? stage : 0) : 3;
      for (int k = 1; k <= kmax; ++k) {
        T2S2_TRY(launch(staged, k));  // warm-up (same result each time)
        T2S2_CUDA_TRY(cudaEventRecord(e0, st));
        T2S2_TRY(launch(staged, k));
        T2S2_TRY(launch(staged, k));
        T2S2_CUDA_TRY(cudaEventRecord(e1, st));
        T2S2_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        T2S2_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        ms *= 0.5f;
        tv.trials.emplace_back(staged, k, ms);
        if (ms < best) best = ms, tv.ctas_per_sm = k, tv.staged = staged;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    it = g_table.emplace(key, tv).first;
  } else {
    T2S2_TRY(launch(it->second.staged, it->second.ctas_per_sm));
  }
  int herr = 0;
  if (tc) T2S2_CUDA_TRY(cudaMemcpyAsync(&herr, g_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  T2S2_CUDA_TRY(cudaStreamSynchronize(st));
  for (int i = 0; i < count; ++i)
    for (int k = 0; k <= ys[i].d; ++k) y[i].r[k] = ys[i].r[k];
  return herr ? T2S2_ETIMEOUT : T2S2_OK;
}

int t2s2_autotune_report(char* buf, int len) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::string s;
  for (auto& kv : g_table) {
    char line[256];
    int o = std::snprintf(line, sizeof(line), "apply prec=%d m<=%d r<=%d tiles<=%d stage<=%ld: %s %d CTAs/SM [",
                          kv.first.prec, kv.first.mb * 16, kv.first.rb, kv.first.tb, kv.first.sb,
                          kv.second.staged ? "staged" : "direct", kv.second.ctas_per_sm);
    s.append(line, std::min<int>(o, (int)sizeof(line) - 1));
    for (auto& t : kv.second.trials) {
      o = std::snprintf(line, sizeof(line), " %s%d:%.4fms", std::get<0>(t) ? "s" : "d", std::get<1>(t),
                        std::get<2>(t));
      s.append(line, std::min<int>(o, (int)sizeof(line) - 1));
    }
    s += " ]\n";
  }
  if (buf && len > 0) {
    const int n = std::min<int>(len - 1, (int)s.size());
    std::memcpy(buf, s.data(), n);
    buf[n] = '\0';
  }
  return (int)s.size();
}

}  // extern "C"

// t2s2_norm_noalloc: the accurate TT norm of t2s2_norm, for callers that may
// not allocate device memory.
//
// Every temporary (the orthogonalised copy of the train, the CholeskyQR
// factors, the split-K partial products, the status word) is carved out of
// one file-scope device array of kNoAllocScratchBytes; no cudaMalloc,
// cudaFree or allocating library call happens on this path.  The array exists
// once per device that loads the library and lives until process exit.
//
// Host code cannot use the array's name as a device address (it is a host-side
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current and caches it.  Because
// that lookup is a CUDA runtime call, the first call on a device should happen
// before any stream capture that wants to record later calls.
//
// All calls share the array: calls whose GPU work overlaps (two streams, two
// host threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "api_internal.h"

namespace t2s2 {

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};
double g_noalloc_host[8];  // pageable host landing slot for the reduction result

// Upper bound of the scratch tt_norm needs for this train: a copy of the
// cores, sized as tt_norm allocates it (every interior core padded to
// max(r_k, rc) x m_k x max(r_{k+1}, rc), rc the largest rank), plus the
// largest per-core orthogonalisation step (LQ factors, the three CholeskyQR
// passes, the neighbour product and split-K partials).
size_t splitk_elems(int M, int N, int K, bool tA, bool tB) {
  Gemm<double> g;
  g.M = M; g.N = N; g.K = K; g.tA = tA; g.tB = tB;
  return gemm_workspace(g);
}

size_t norm_scratch_bytes(const DevTT& x) {
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  int rc = 0;
  for (int k = 0; k <= x.d; ++k) rc = std::max(rc, x.r[k]);
  size_t copy = 0;
  for (int k = 0; k < x.d; ++k) {
    const size_t r0 = (k == 0) ? 1 : std::max(x.r[k], rc);
    const size_t r1 = (k == x.d - 1) ? 1 : std::max(x.r[k + 1], rc);
    copy += al(r0 * x.m[k] * r1 * sizeof(double));
  }
  size_t step = 0;
  for (int k = x.d - 1; k >= 1; --k) {
    const int rk = x.r[k], cols = x.m[k] * x.r[k + 1];
    const int prev = x.r[k - 1] * x.m[k - 1];
    const int nb = std::max(rk, cols);
    size_t ws = 0;  // largest split-K partial buffer among the step's GEMMs
    ws = std::max(ws, splitk_elems(rk, rk, cols, false, true));   // Gram
    ws = std::max(ws, splitk_elems(rk, cols, rk, false, false));  // L^{-1} W
    ws = std::max(ws, splitk_elems(rk, rk, rk, false, false));    // factor product
    ws = std::max(ws, splitk_elems(prev, nb, rk, false, false));  // neighbour core
    const size_t s = 3 * al((size_t)rk * cols * 8) + al((size_t)prev * nb * 8) +
                     8 * al((size_t)rk * rk * 8) + al(ws * 8);
    step = std::max(step, s);
  }
  return copy + step + ((size_t)64 << 10);
}

t2s2_status scratch_address(void** out) {
  int dev = -1;
  T2S2_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return T2S2_ENODEV;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      return T2S2_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return T2S2_OK;
}

}  // namespace
}  // namespace t2s2

using namespace t2s2;

extern "C" {

t2s2_status t2s2_norm_noalloc(const t2s2_tt* x, double* out, void* stream) {
  if (!x || !out || !x->r || !x->cores || !x->cap || !x->m) return T2S2_EINVAL;
  if (x->d < 1 || x->d > T2S2_MAX_D || x->loc != T2S2_DEVICE) return T2S2_EINVAL;
  if (x->r[0] != 1 || x->r[x->d] != 1) return T2S2_EINVAL;
  DevTT dv;
  dv.d = x->d;
  for (int k = 0; k <= x->d; ++k) dv.r[k] = x->r[k];
  for (int k = 0; k < x->d; ++k) {
    if (x->m[k] < 1 || x->r[k + 1] < 1 || !x->cores[k]) return T2S2_EINVAL;
    if (x->r[k] > kSmallMax) return T2S2_EINVAL;
    dv.m[k] = x->m[k];
    dv.c[k] = x->cores[k];
    dv.cap[k] = x->cap[k];
    if (dv.core_elems(k) > x->cap[k]) return T2S2_ENOMEM;
  }
  // Reject trains whose temporaries would not fit the static array.
  if (norm_scratch_bytes(dv) > kNoAllocScratchBytes) return T2S2_ENOMEM;
  void* base = nullptr;
  T2S2_TRY(scratch_address(&base));
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  Arena ar;
  ar.base = static_cast<char*>(base);
  ar.size = kNoAllocScratchBytes;
  Ctx cx;
  cx.st = static_cast<cudaStream_t>(stream);
  cx.ar = &ar;
  cx.hbuf = g_noalloc_host;
  cx.dstat = aget<int>(cx, 64);
  if (!cx.dstat) return T2S2_ENOMEM;
  // the status word must start at zero on every call (the array keeps the
  // previous call's contents)
  T2S2_CUDA_TRY(cudaMemsetAsync(cx.dstat, 0, 64 * sizeof(int), cx.st));
  const t2s2_status st = tt_norm(cx, dv, out);
  // On an error part of the work may still be queued on the array: let it
  // finish before the next caller can take the lock.
  if (st != T2S2_OK) (void)cudaStreamSynchronize(cx.st);
  return st;
}

}  // extern "C"

// Test driver (CPU only: it launches nothing): prints, one per line, the
// small-GEMM plan that the library's latency model picks for each shape read
// from stdin ("M N K batch" per line), as "use bm bn splits kc".  The planner
// lives in an anonymous namespace of gemm.cu, so that file is included here.
#include <cstdio>

#include "../../paper_2506_04732_gb300/csrc/gemm.cu"

int main() {
  long M, N, K, batch;
  while (std::scanf("%ld %ld %ld %ld", &M, &N, &K, &batch) == 4) {
    t2s2::Gemm<double> g{};
    g.M = (int)M;
    g.N = (int)N;
    g.K = (int)K;
    g.batch = (int)batch;
    const auto p = t2s2::plan_small(g);
    std::printf("%d %d %d %d %d\n", p.use ? 1 : 0, p.bm, p.bn, p.splits, p.kc);
  }
  return 0;
}

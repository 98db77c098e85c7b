// Test driver (CPU only: it launches nothing) for the small-GEMM planners of
// gemm.cu, which live in an anonymous namespace, so that file is included.
// stdin, one request per line:
//   "s M N K batch"            -> "use bm bn splits kc"           (plan_small)
//   "g n M N K batch ... (n x)" -> "ok bm bn splits_0 kc_0 ..."   (plan_group)
#include <cstdio>

#include "../../paper_2506_04732_gb300/csrc/gemm.cu"

static bool read_gemm(t2s2::Gemm<double>* g) {
  long M, N, K, batch;
  if (std::scanf("%ld %ld %ld %ld", &M, &N, &K, &batch) != 4) return false;
  *g = t2s2::Gemm<double>{};
  g->M = (int)M;
  g->N = (int)N;
  g->K = (int)K;
  g->batch = (int)batch;
  return true;
}

int main() {
  char kind[4];
  while (std::scanf("%3s", kind) == 1) {
    if (kind[0] == 's') {
      t2s2::Gemm<double> g;
      if (!read_gemm(&g)) return 1;
      const auto p = t2s2::plan_small(g);
      std::printf("%d %d %d %d %d\n", p.use ? 1 : 0, p.bm, p.bn, p.splits, p.kc);
    } else {
      int n = 0;
      if (std::scanf("%d", &n) != 1 || n < 1 || n > t2s2::kMaxGroup) return 1;
      t2s2::Gemm<double> gs[t2s2::kMaxGroup];
      for (int i = 0; i < n; ++i)
        if (!read_gemm(&gs[i])) return 1;
      const auto p = t2s2::plan_group(gs, n);
      std::printf("%d %d %d", p.ok ? 1 : 0, p.bm, p.bn);
      for (int i = 0; i < n; ++i) std::printf(" %d %d", p.ok ? p.splits[i] : 0, p.ok ? p.kc[i] : 0);
      std::printf("\n");
    }
  }
  return 0;
}

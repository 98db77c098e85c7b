// Test driver (CPU): prints, as JSON, the library's host-side data of one
// dimension -- B = Rt^{-1} Lt and its complex Schur form B = Z T Z^H -- so
// that a Python test can check them against numpy and the oracle.
// Usage: host_1d_check n eps beta plain     (a space dimension)
//        host_1d_check time n scale          (the time dimension of the space-time form)
#include <cstdio>
#include <cstdlib>

#include "../../paper_2506_04732_gb300/csrc/host_1d.h"

static void put(const char* name, const std::vector<double>& v, bool last = false) {
  std::printf("\"%s\": [", name);
  for (size_t i = 0; i < v.size(); ++i) std::printf("%s%.17g", i ? ", " : "", v[i]);
  std::printf("]%s\n", last ? "" : ",");
}

int main(int argc, char** argv) {
  t2s2::Dim1D D;
  const bool time = argc == 4 && argv[1][0] == 't';
  if (!time && argc != 5) return 2;
  const bool ok = time ? t2s2::build_time_dimension(std::atoi(argv[2]), std::atof(argv[3]), &D)
                       : t2s2::build_dimension(std::atoi(argv[1]), std::atof(argv[2]), std::atof(argv[3]),
                                               std::atoi(argv[4]), &D);
  if (!ok) return 1;
  std::printf("{\n");
  put("x", D.x);
  put("eta", D.eta);
  if (time) {
    put("R0", D.R0);
    put("L0", D.L0);
  }
  put("Rt", D.Rt);
  put("Lt", D.Lt);
  put("Rinv", D.Rinv);
  put("B", D.B);
  put("Tr", D.Tr);
  put("Ti", D.Ti);
  put("Zr", D.Zr);
  put("Zi", D.Zi, true);
  std::printf("}\n");
  return 0;
}

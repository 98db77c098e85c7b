// Local solves of the alternating TT solver (see local.cu).
#pragma once
#include "common.cuh"

namespace t2s2 {

constexpr int kLocalMaxM = 128;        // largest mode size handled by the local solver
constexpr int kLocalMaxRestart = 40;   // largest GMRES restart length
constexpr int kLocalTimingIts = 12;
constexpr int kLocalOwnMax = 4096;     // own-element index list kept in shared memory up to this size    // iterations covered by the optional phase timestamps

template <typename T>
struct LocalProblem {
  int ra = 0, m = 0, rb = 0;           // local core shape; N = ra * m * rb
  const double* PL = nullptr;          // ra x ra left interface (Kronecker-sum part)
  const double* PR = nullptr;          // rb x rb right interface
  const double* Bp = nullptr;          // m x m  B' = c_op B + shift I
  const float *Tr = nullptr, *Ti = nullptr, *Zr = nullptr, *Zi = nullptr;  // Schur B = Z T Z^H (binary32)
  double c_op = 1.0, shift = 0.0;
  const T* rhs = nullptr;              // N
  T* x = nullptr;                      // N, initial guess in, solution out
  T* work = nullptr;                   // local_work_elems(N, mr)
  double* part = nullptr;              // 2 * team * (kLocalMaxRestart + 2)
  double tol_rel = 1e-10;              // stop at ||rhs - K x|| <= tol_rel ||rhs||
  int maxit = 400, mr = 30, team = 0;  // team = 0: pick the number of CTAs
  const float *Ttc_r = nullptr, *Ttc_i = nullptr;  // (c_op T)^T in global memory when m is too big for smem
  int smem_mats = 0;                   // set by the launcher
  int own_cap = 0;                     // set by the launcher: own-element indices kept in smem
  int fls = 0;                         // 1: exact Kronecker-sum preconditioner (needs the buffers below)
  void* eigL = nullptr;                // complex binary32: lam[ra], V[ra*ra], Vinv[ra*ra]
  void* eigR = nullptr;                // complex binary32: lam[rb], V[rb*rb], Vinv[rb*rb]
  int* eig_status = nullptr;           // 2 ints written by the eigendecomposition kernel
  void* ybuf = nullptr;                // N complex binary32 values
  unsigned long long* tstamp = nullptr;  // optional phase timestamps (diagnostics)
  int* iters_out = nullptr;            // total GMRES iterations
  double* res_out = nullptr;           // [final residual norm, ||rhs||]
  const int* skip = nullptr;           // device word: 0 = solved already, return at once
};

// Local solve with rb = 1 in one CTA (sylv.cu): binary64 refinement around
// the Schur-basis Sylvester solver in binary32.  *status = 0 when ||rhs - K x||
// <= tol_rel ||rhs||, else 1 with the iterate left in x.
struct SylvProblem {
  int ra = 0, m = 0;
  const double* PL = nullptr;          // ra x ra
  const double* PR = nullptr;          // 1 x 1
  const double* Bp = nullptr;          // m x m  B' = c_op B + shift I
  const float *Tr = nullptr, *Ti = nullptr, *Zr = nullptr, *Zi = nullptr;  // Schur B = Z T Z^H
  double c_op = 1.0, shift = 0.0;
  const double* rhs = nullptr;         // ra x m
  double* x = nullptr;                 // ra x m, initial guess in, iterate out
  double tol_rel = 1e-10;
  int* status = nullptr;
  int* iters_out = nullptr;
  double* res_out = nullptr;
  unsigned long long* tstamp = nullptr;  // optional phase timestamps (diagnostics), kSylvStamps slots
};
constexpr int kSylvStamps = 48;
bool sylv_rb1_fits(int ra, int m);
t2s2_status sylv_rb1(const SylvProblem& P, cudaStream_t st);

template <typename T>
size_t local_work_elems(long N, int mr);

constexpr size_t kLocalSmemCap = 200 * 1024;
constexpr size_t kLocalPartElems = 2 * 160 * (kLocalMaxRestart + 2);

// Algorithmic FLOPs of one local GMRES solve that took `its` iterations.
double local_flops(int ra, int m, int rb, int its, int mr);

template <typename T>
t2s2_status local_gmres(const LocalProblem<T>& P, cudaStream_t st);

}  // namespace t2s2

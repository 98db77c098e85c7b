// Eigendecomposition A = V diag(lam) V^{-1} of a small real nonsymmetric
// matrix (r <= kEigMax) by one warp in shared memory, complex binary32.
//
// Steps (all unitary until the last one):
//   1. Householder reduction to upper Hessenberg form, H = U^T A U;
//   2. complex single-shift QR sweeps on H (Givens bulge chasing, Wilkinson
//      shifts, deflation of negligible subdiagonals): H = Q T Q^H, U <- U Q;
//   3. eigenvectors of the triangular T by back substitution, X upper
//      triangular with unit diagonal (tiny pivots are replaced by eps ||T||);
//   4. V = U X D with D normalising the columns, V^{-1} = D^{-1} X^{-1} U^H.
// The decomposition feeds a preconditioner: its accuracy sets how fast the
// outer Krylov solver converges, not the accuracy of the solution.
#pragma once
#include <cuda_runtime.h>

namespace t2s2 {

constexpr int kEigMax = 64;

struct cf {
  float x, y;
};
__device__ __forceinline__ cf cmk(float a, float b) { return cf{a, b}; }
__device__ __forceinline__ cf cadd(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cf csub(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cf cmul(cf a, cf b) { return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cf cconj(cf a) { return cf{a.x, -a.y}; }
__device__ __forceinline__ float cabs2(cf a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float cabsf(cf a) { return hypotf(a.x, a.y); }
__device__ __forceinline__ cf cscale(cf a, float s) { return cf{a.x * s, a.y * s}; }
__device__ __forceinline__ cf cdiv(cf a, cf b) {
  const float d = __frcp_rn(cabs2(b));
  return cf{(a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d};
}
__device__ __forceinline__ cf csqrtf(cf a) {
  const float r = cabsf(a);
  if (r == 0.f) return cf{0.f, 0.f};
  float re = sqrtf(0.5f * (r + fabsf(a.x)));
  float im = 0.5f * a.y / re;
  if (a.x >= 0.f) return cf{re, im};
  return cf{fabsf(im), copysignf(re, a.y)};
}
__device__ __forceinline__ float wsum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory workspace for one decomposition: three r x (r+1) complex
// matrices and two length-r vectors (eig_smem_bytes(r) bytes).
struct EigSmem {
  cf* T;
  cf* U;
  cf* X;
  float* v;
  float* scale;
  int ld;
};
__host__ __device__ inline size_t eig_smem_bytes(int r) {
  return (size_t)3 * r * (r + 1) * sizeof(cf) + (size_t)2 * r * sizeof(float);
}
__device__ inline EigSmem eig_smem(void* base, int r) {
  EigSmem e;
  e.ld = r + 1;
  e.T = reinterpret_cast<cf*>(base);
  e.U = e.T + r * e.ld;
  e.X = e.U + r * e.ld;
  e.v = reinterpret_cast<float*>(e.X + r * e.ld);
  e.scale = e.v + r;
  return e;
}

// Executed by one full warp.  A: r x r row-major (leading dimension lda), any
// precision convertible to float.  Outputs (global or shared, row-major r x r):
// lam[r], V, Vinv.  Returns false if the QR iteration did not converge.
template <typename TA>
__device__ bool warp_eig(const TA* A, int lda, int r, EigSmem& s, cf* lam, cf* V, int ldv, cf* Vinv,
                         int ldvi) {
  const int lane = threadIdx.x & 31;
  const int ld = s.ld;
  auto t = [&](int i, int j) -> cf& { return s.T[i * ld + j]; };
  auto u = [&](int i, int j) -> cf& { return s.U[i * ld + j]; };
  auto x = [&](int i, int j) -> cf& { return s.X[i * ld + j]; };
  for (int e = lane; e < r * r; e += 32) {
    const int i = e / r, j = e % r;
    t(i, j) = cmk((float)A[(long)i * lda + j], 0.f);
    u(i, j) = cmk(i == j ? 1.f : 0.f, 0.f);
  }
  __syncwarp();
  // 1. Householder reduction to Hessenberg form (real arithmetic on .x)
  for (int k = 0; k + 2 < r; ++k) {
    float a2 = 0.f;
    for (int i = k + 1 + lane; i < r; i += 32) a2 += t(i, k).x * t(i, k).x;
    a2 = wsum(a2);
    if (a2 == 0.f) continue;
    const float alpha = sqrtf(a2);
    const float x0 = t(k + 1, k).x;
    const float sg = (x0 >= 0.f) ? -alpha : alpha;
    for (int i = lane; i < r; i += 32) s.v[i] = (i == k + 1) ? x0 - sg : ((i > k + 1) ? t(i, k).x : 0.f);
    __syncwarp();
    float vn = 0.f;
    for (int i = k + 1 + lane; i < r; i += 32) vn += s.v[i] * s.v[i];
    vn = wsum(vn);
    if (vn == 0.f) continue;
    const float tau = 2.f / vn;
    for (int j = k + lane; j < r; j += 32) {  // left: rows k+1..r-1
      float sm = 0.f;
      for (int i = k + 1; i < r; ++i) sm += s.v[i] * t(i, j).x;
      sm *= tau;
      for (int i = k + 1; i < r; ++i) t(i, j).x -= sm * s.v[i];
    }
    __syncwarp();
    for (int i = lane; i < r; i += 32) {  // right: columns k+1..r-1, and U <- U P
      float sm = 0.f, su = 0.f;
      for (int j = k + 1; j < r; ++j) {
        sm += t(i, j).x * s.v[j];
        su += u(i, j).x * s.v[j];
      }
      sm *= tau;
      su *= tau;
      for (int j = k + 1; j < r; ++j) {
        t(i, j).x -= sm * s.v[j];
        u(i, j).x -= su * s.v[j];
      }
    }
    __syncwarp();
    for (int i = k + 2 + lane; i < r; i += 32) t(i, k).x = 0.f;
    __syncwarp();
  }
  // 2. complex single-shift QR on the Hessenberg matrix
  float tnorm = 0.f;
  for (int e = lane; e < r * r; e += 32) tnorm = fmaxf(tnorm, cabsf(t(e / r, e % r)));
  for (int o = 16; o > 0; o >>= 1) tnorm = fmaxf(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  const float eps = 1.2e-7f;
  int hi = r - 1, iter = 0, total = 0;
  bool ok = true;
  while (hi > 0) {
    // the largest l <= hi whose subdiagonal is negligible relative to its
    // diagonal neighbours or, norm-wise, to the matrix (a backward-stable
    // perturbation of eps ||T||; tiny eigenvalues otherwise wait for a
    // relative test that binary32 noise never lets them pass); 0 if none.
    // Lanes test l = lane + 1 + 32 c in parallel, a ballot picks the largest.
    int l = 0;
    for (int c0 = ((hi - 1) / 32) * 32; c0 >= 0 && l == 0; c0 -= 32) {
      const int li = c0 + lane + 1;
      bool neg = false;
      if (li <= hi) {
        const float sub = sqrtf(cabs2(t(li, li - 1)));
        const float dg = sqrtf(cabs2(t(li - 1, li - 1))) + sqrtf(cabs2(t(li, li)));
        neg = sub <= eps * fmaxf(dg, tnorm);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, neg);
      if (mask) l = c0 + 32 - __clz(mask);
    }
    __syncwarp();
    if (l > 0 && lane == 0) t(l, l - 1) = cmk(0.f, 0.f);
    __syncwarp();
    if (l == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * r) {
      ok = false;
      break;
    }
    ++iter;
    cf mu;
    if (iter % 11 == 0) {
      mu = cadd(t(hi, hi), cmk(0.75f * cabsf(t(hi, hi - 1)), 0.f));
    } else {
      const cf a = t(hi - 1, hi - 1), b = t(hi - 1, hi), c = t(hi, hi - 1), d = t(hi, hi);
      const cf half = cscale(csub(a, d), 0.5f);
      const cf disc = csqrtf(cadd(cmul(half, half), cmul(b, c)));
      const cf mid = cscale(cadd(a, d), 0.5f);
      const cf l1 = cadd(mid, disc), l2 = csub(mid, disc);
      mu = (cabs2(csub(l1, d)) < cabs2(csub(l2, d))) ? l1 : l2;
    }
    cf xx = csub(t(l, l), mu), yy = t(l + 1, l);
    for (int k = l; k < hi; ++k) {
      // rotation [c, s; -conj(s), c] with c = |x| / r, s = (x / |x|) conj(y) / r,
      // r = sqrt(|x|^2 + |y|^2), from binary32 reciprocal square roots
      const float nx = cabs2(xx), ny = cabs2(yy), n2 = nx + ny;
      float c;
      cf sn;
      if (n2 == 0.f) {
        c = 1.f;
        sn = cmk(0.f, 0.f);
      } else if (nx == 0.f) {
        c = 0.f;
        sn = cscale(cconj(yy), rsqrtf(ny));
      } else {
        const float ix = rsqrtf(nx), ir = rsqrtf(n2);
        c = nx * ix * ir;
        sn = cscale(cmul(cscale(xx, ix), cconj(yy)), ir);
      }
      const cf sbar = cconj(sn);
      for (int j = (k - 1 > l ? k - 1 : l) + lane; j < r; j += 32) {
        const cf p = t(k, j), q = t(k + 1, j);
        t(k, j) = cadd(cscale(p, c), cmul(sn, q));
        t(k + 1, j) = csub(cscale(q, c), cmul(sbar, p));
      }
      __syncwarp();
      const int rmax = (k + 2 < hi) ? k + 2 : hi;
      for (int i = lane; i <= rmax; i += 32) {
        const cf p = t(i, k), q = t(i, k + 1);
        t(i, k) = cadd(cscale(p, c), cmul(sbar, q));
        t(i, k + 1) = csub(cscale(q, c), cmul(sn, p));
      }
      for (int i = lane; i < r; i += 32) {
        const cf p = u(i, k), q = u(i, k + 1);
        u(i, k) = cadd(cscale(p, c), cmul(sbar, q));
        u(i, k + 1) = csub(cscale(q, c), cmul(sn, p));
      }
      __syncwarp();
      if (k + 2 <= hi) {
        xx = t(k + 1, k);
        yy = t(k + 2, k);
      }
    }
  }
  __syncwarp();
  // 3. eigenvectors of the triangular T: column k of X, lane-parallel over k
  const float small = eps * (tnorm > 0.f ? tnorm : 1.f);
  for (int k = lane; k < r; k += 32) {
    const cf lk = t(k, k);
    for (int i = r - 1; i > k; --i) x(i, k) = cmk(0.f, 0.f);
    x(k, k) = cmk(1.f, 0.f);
    for (int i = k - 1; i >= 0; --i) {
      cf sm = cmk(0.f, 0.f);
      for (int l2 = i + 1; l2 <= k; ++l2) sm = cadd(sm, cmul(t(i, l2), x(l2, k)));
      cf den = csub(t(i, i), lk);
      if (cabsf(den) < small) den = cmk(small, 0.f);
      x(i, k) = cdiv(cscale(sm, -1.f), den);
    }
  }
  __syncwarp();
  // 4. V = U X D, D normalises columns; V^{-1} = D^{-1} X^{-1} U^H
  for (int k = lane; k < r; k += 32) {
    float nrm = 0.f;
    for (int i = 0; i < r; ++i) {
      cf sm = cmk(0.f, 0.f);
      for (int l2 = 0; l2 <= k; ++l2) sm = cadd(sm, cmul(u(i, l2), x(l2, k)));
      nrm += cabs2(sm);
    }
    s.scale[k] = (nrm > 0.f) ? rsqrtf(nrm) : 1.f;
    lam[k] = t(k, k);
  }
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    const int i = e / r, k = e % r;
    cf sm = cmk(0.f, 0.f);
    for (int l2 = 0; l2 <= k; ++l2) sm = cadd(sm, cmul(u(i, l2), x(l2, k)));
    V[(long)i * ldv + k] = cscale(sm, s.scale[k]);
  }
  __syncwarp();
  // X^{-1} (upper triangular, unit diagonal) into T's storage, lane per column
  for (int k = lane; k < r; k += 32) {
    for (int i = r - 1; i > k; --i) t(i, k) = cmk(0.f, 0.f);
    t(k, k) = cmk(1.f, 0.f);
    for (int i = k - 1; i >= 0; --i) {
      cf sm = cmk(0.f, 0.f);
      for (int l2 = i + 1; l2 <= k; ++l2) sm = cadd(sm, cmul(x(i, l2), t(l2, k)));
      t(i, k) = cscale(sm, -1.f);
    }
  }
  __syncwarp();
  for (int e = lane; e < r * r; e += 32) {
    const int k = e / r, j = e % r;  // row k of D^{-1} X^{-1} U^H
    cf sm = cmk(0.f, 0.f);
    for (int l2 = k; l2 < r; ++l2) sm = cadd(sm, cmul(t(k, l2), cconj(u(j, l2))));
    Vinv[(long)k * ldvi + j] = cscale(sm, 1.f / s.scale[k]);
  }
  __syncwarp();
  return ok;
}

}  // namespace t2s2

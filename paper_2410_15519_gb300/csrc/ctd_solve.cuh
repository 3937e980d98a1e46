// Banded SPD solve of one fixed-point half-sweep (Eq. ux): (a1 diag(omega) + a2 K) y = q.
//
// One CTA.  The matrix has half bandwidth b (= 2s+1), so with blocks of b rows it is block
// tridiagonal.  It is factorised in FP32 by block cyclic reduction (odd blocks of the active
// set are eliminated level by level; log2(n/b) levels of independent block operations), and
// the FP32 solution is refined with residuals computed in double-float arithmetic
// (48-bit significand) until the correction falls below 2^-47 of the iterate, which brings
// the result to FP64-level accuracy.  Native FP64 is avoided: on this part it runs at about
// 1/60 of the FP32 rate with a 64-cycle dependent latency.
#pragma once
#include "ctd_common.cuh"

namespace ctd {

// Compressed stiffness: rows [0, nlead) and [n - ntail, n) stored explicitly, every other row
// equals the interior stencil (uniform mesh: all interior elements share one element matrix).
struct KCompressed {
  int n, b, nlead, ntail;
  const float2* rows;      // [(nlead + ntail)][2b+1] double-float
  const float2* stencil;   // [2b+1]
  float2 omega_in, omega_end;   // nodal weights inside / at the two ends
};

__device__ __forceinline__ float2 kc_entry(const KCompressed& k, int i, int off /* -b..b */) {
  const int w = 2 * k.b + 1;
  if (i < k.nlead) return k.rows[i * w + off + k.b];
  if (i >= k.n - k.ntail) return k.rows[(k.nlead + i - (k.n - k.ntail)) * w + off + k.b];
  return k.stencil[off + k.b];
}
__device__ __forceinline__ float2 kc_omega(const KCompressed& k, int i) {
  return (i == 0 || i == k.n - 1) ? k.omega_end : k.omega_in;
}

struct CRBuffers {
  float *D, *E, *G1, *G2;  // [nb][b*b]
  float *F, *Y, *X;        // [nb*b]
  int nb, b;
};

__host__ __device__ inline size_t cr_floats(int n, int b) {
  const int nb = (n + b - 1) / b;
  return static_cast<size_t>(nb) * b * b * 4 + static_cast<size_t>(nb) * b * 3;
}

__device__ inline CRBuffers cr_bind(float* base, int n, int b) {
  CRBuffers s;
  s.b = b;
  s.nb = (n + b - 1) / b;
  const size_t bs = static_cast<size_t>(s.nb) * b * b;
  s.D = base;
  s.E = base + bs;
  s.G1 = base + 2 * bs;
  s.G2 = base + 3 * bs;
  s.F = base + 4 * bs;
  s.Y = s.F + s.nb * b;
  s.X = s.Y + s.nb * b;
  return s;
}

// Cholesky L L^T of a b x b row-major block, in place (lower triangle).  Returns false if a
// pivot is not positive.
__device__ inline bool chol_block(float* A, int b) {
  bool ok = true;
  for (int j = 0; j < b; ++j) {
    float d = A[j * b + j];
    for (int k = 0; k < j; ++k) d -= A[j * b + k] * A[j * b + k];
    if (!(d > 0.f)) { ok = false; d = 1.f; }
    d = sqrtf(d);
    A[j * b + j] = d;
    const float inv = 1.f / d;
    for (int i = j + 1; i < b; ++i) {
      float v = A[i * b + j];
      for (int k = 0; k < j; ++k) v -= A[i * b + k] * A[j * b + k];
      A[i * b + j] = v * inv;
    }
  }
  return ok;
}

// x <- (L L^T)^-1 x for a vector with stride sx
__device__ inline void chol_apply(const float* L, int b, float* x, int sx) {
  for (int i = 0; i < b; ++i) {
    float v = x[i * sx];
    for (int k = 0; k < i; ++k) v -= L[i * b + k] * x[k * sx];
    x[i * sx] = v / L[i * b + i];
  }
  for (int i = b - 1; i >= 0; --i) {
    float v = x[i * sx];
    for (int k = i + 1; k < b; ++k) v -= L[k * b + i] * x[k * sx];
    x[i * sx] = v / L[i * b + i];
  }
}

// Fill D (diagonal blocks) and E (E[I] = rows of block I+1, columns of block I) of
// a1 diag(omega) + a2 K in FP32; rows past n are identity.
__device__ inline void cr_build(const CRBuffers& s, const KCompressed& k, float a1, float a2) {
  const int b = s.b, bsz = b * b, n = k.n;
  for (int t = threadIdx.x; t < s.nb * bsz; t += blockDim.x) {
    const int I = t / bsz, e = t - I * bsz, r = e / b, c = e - r * b;
    const int row = I * b + r, col = I * b + c;
    float dv;
    if (row < n && col < n) {
      dv = a2 * kc_entry(k, row, col - row).x;
      if (row == col) dv += a1 * kc_omega(k, row).x;
    } else {
      dv = (r == c) ? 1.f : 0.f;
    }
    s.D[t] = dv;
    const int row2 = row + b;
    float ev = 0.f;
    if (I + 1 < s.nb && row2 < n && col < n && row2 - col <= b) ev = a2 * kc_entry(k, row2, col - row2).x;
    s.E[t] = ev;
  }
}

// Block cyclic reduction factorisation.  Returns false if a pivot failed.
__device__ inline bool cr_factor(const CRBuffers& s) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  const int b = s.b, bsz = b * b;
  int st = 1, K = s.nb;
  while (K > 1) {
    const int nodd = K / 2, neven = (K + 1) / 2;
    for (int q = threadIdx.x; q < nodd; q += blockDim.x) {
      const int j = (2 * q + 1) * st;
      if (!chol_block(s.D + j * bsz, b)) s_ok = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nodd * 2 * b; t += blockDim.x) {
      const int q = t / (2 * b), col = t - q * 2 * b, k = 2 * q + 1, j = k * st;
      const float* L = s.D + j * bsz;
      if (col < b) {               // G1[j] = D_j^-1 E[j-st]   (couples j to j-st)
        float* g = s.G1 + j * bsz + col;
        const float* e = s.E + (j - st) * bsz + col;
        for (int r = 0; r < b; ++r) g[r * b] = e[r * b];
        chol_apply(L, b, g, b);
      } else {                     // G2[j] = D_j^-1 E[j]^T    (couples j to j+st)
        const int c = col - b;
        float* g = s.G2 + j * bsz + c;
        if (k + 1 < K) {
          const float* e = s.E + j * bsz + c * b;   // row c of E[j]
          for (int r = 0; r < b; ++r) g[r * b] = e[r];
          chol_apply(L, b, g, b);
        } else {
          for (int r = 0; r < b; ++r) g[r * b] = 0.f;
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < neven * bsz; t += blockDim.x) {
      const int q = t / bsz, e = t - q * bsz, r = e / b, c = e - r * b, k = 2 * q, i = k * st;
      float acc = s.D[i * bsz + e];
      if (k >= 1) {                // left odd neighbour j = i - st: E[j] G2[j]
        const int j = i - st;
        for (int l = 0; l < b; ++l) acc -= s.E[j * bsz + r * b + l] * s.G2[j * bsz + l * b + c];
      }
      if (k + 1 < K) {             // right odd neighbour j = i + st: E[i]^T G1[j]
        const int j = i + st;
        for (int l = 0; l < b; ++l) acc -= s.E[i * bsz + l * b + r] * s.G1[j * bsz + l * b + c];
      }
      s.D[i * bsz + e] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < neven * bsz; t += blockDim.x) {
      const int q = t / bsz, e = t - q * bsz, r = e / b, c = e - r * b, k = 2 * q, i = k * st;
      if (k + 2 < K) {             // new coupling i <-> i + 2st: -E[j] G1[j], j = i + st
        const int j = i + st;
        float acc = 0.f;
        for (int l = 0; l < b; ++l) acc -= s.E[j * bsz + r * b + l] * s.G1[j * bsz + l * b + c];
        s.E[i * bsz + e] = acc;
      }
    }
    __syncthreads();
    st *= 2;
    K = (K + 1) / 2;
  }
  if (threadIdx.x == 0 && !chol_block(s.D, b)) s_ok = 0;
  __syncthreads();
  return s_ok != 0;
}

// Solve with the factors; right-hand side in s.F (nb*b, padded rows zero), result in s.X.
__device__ inline void cr_solve(const CRBuffers& s) {
  const int b = s.b, bsz = b * b;
  int st = 1, K = s.nb, levels = 0;
  while (K > 1) {
    const int nodd = K / 2, neven = (K + 1) / 2;
    for (int q = threadIdx.x; q < nodd; q += blockDim.x) {
      const int j = (2 * q + 1) * st;
      for (int r = 0; r < b; ++r) s.Y[j * b + r] = s.F[j * b + r];
      chol_apply(s.D + j * bsz, b, s.Y + j * b, 1);
    }
    for (int t = threadIdx.x; t < neven * b; t += blockDim.x) {
      const int q = t / b, r = t - q * b, k = 2 * q, i = k * st;
      float acc = s.F[i * b + r];
      if (k >= 1) {
        const int j = i - st;
        for (int l = 0; l < b; ++l) acc -= s.G2[j * bsz + l * b + r] * s.F[j * b + l];
      }
      if (k + 1 < K) {
        const int j = i + st;
        for (int l = 0; l < b; ++l) acc -= s.G1[j * bsz + l * b + r] * s.F[j * b + l];
      }
      s.Y[i * b + r] = acc;      // stage the update, copied back below (F of odd j still read)
    }
    __syncthreads();
    for (int t = threadIdx.x; t < neven * b; t += blockDim.x) {
      const int q = t / b, r = t - q * b, i = 2 * q * st;
      s.F[i * b + r] = s.Y[i * b + r];
    }
    __syncthreads();
    st *= 2;
    K = (K + 1) / 2;
    ++levels;
  }
  if (threadIdx.x == 0) {
    for (int r = 0; r < b; ++r) s.X[r] = s.F[r];
    chol_apply(s.D, b, s.X, 1);
  }
  __syncthreads();
  for (int lv = levels - 1; lv >= 0; --lv) {
    st = 1 << lv;
    K = (s.nb + st - 1) / st;
    const int nodd = K / 2;
    for (int t = threadIdx.x; t < nodd * b; t += blockDim.x) {
      const int q = t / b, r = t - q * b, k = 2 * q + 1, j = k * st;
      float acc = s.Y[j * b + r];
      for (int l = 0; l < b; ++l) acc -= s.G1[j * bsz + r * b + l] * s.X[(j - st) * b + l];
      if (k + 1 < K)
        for (int l = 0; l < b; ++l) acc -= s.G2[j * bsz + r * b + l] * s.X[(j + st) * b + l];
      s.X[j * b + r] = acc;
    }
    __syncthreads();
  }
}

// Deterministic CTA max of a non-negative value.
__device__ inline float cta_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
  __syncthreads();
  return m;
}

// Full solve with refinement.  q: double-float right-hand side [n]; x: double-float result
// [n] (shared memory).  a1, a2 as double-float.  Returns false on a failed pivot or a
// non-finite result.
__device__ inline bool banded_solve(const CRBuffers& s, const KCompressed& k, dfloat a1,
                                    dfloat a2, const float2* q, float2* x, float* red) {
  const int n = k.n, b = k.b, npad = s.nb * b;
  cr_build(s, k, a1.hi, a2.hi);
  __syncthreads();
  bool ok = cr_factor(s);
  for (int i = threadIdx.x; i < npad; i += blockDim.x) s.F[i] = (i < n) ? q[i].x : 0.f;
  __syncthreads();
  cr_solve(s);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = make_float2(s.X[i], 0.f);
  __syncthreads();
  for (int it = 0; it < 4; ++it) {
    // r = q - (a1 omega x + a2 K x) in double-float
    float rmax = 0.f;
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
      if (i >= n) { s.F[i] = 0.f; continue; }
      dfloat kx = {0.f, 0.f};
      const int j0 = max(0, i - b), j1 = min(n - 1, i + b);
      for (int j = j0; j <= j1; ++j) {
        const float2 kij = kc_entry(k, i, j - i);
        kx = df_fma(kx, dfloat{kij.x, kij.y}, dfloat{x[j].x, x[j].y});
      }
      const float2 om = kc_omega(k, i);
      dfloat ax = df_add(df_mul(a2, kx), df_mul(a1, df_mul(dfloat{om.x, om.y}, dfloat{x[i].x, x[i].y})));
      dfloat r = df_add(dfloat{q[i].x, q[i].y}, df_neg(ax));
      s.F[i] = r.hi + r.lo;
      rmax = fmaxf(rmax, fabsf(r.hi));
    }
    __syncthreads();
    cr_solve(s);
    float dmax = 0.f, xmax = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const dfloat nx = df_add(dfloat{x[i].x, x[i].y}, dfloat{s.X[i], 0.f});
      x[i] = make_float2(nx.hi, nx.lo);
      dmax = fmaxf(dmax, fabsf(s.X[i]));
      xmax = fmaxf(xmax, fabsf(nx.hi));
    }
    dmax = cta_max(dmax, red);
    xmax = cta_max(xmax, red);
    (void)rmax;
    if (!(dmax == dmax) || !(xmax <= 3.0e38f)) return false;   // NaN / Inf
    if (dmax <= 7.105427357601002e-15f * xmax) break;          // 2^-47
  }
  return ok;
}

}  // namespace ctd

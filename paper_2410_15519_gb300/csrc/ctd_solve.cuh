// Banded SPD solve of one fixed-point half-sweep (Eq. ux): (a1 diag(omega) + a2 K) y = q.
//
// One CTA.  The matrix has half bandwidth b (= 2s+1), so with blocks of b rows it is block
// tridiagonal.  It is factorised in FP32 by block cyclic reduction (odd blocks of the active
// set are eliminated level by level; log2(n/b) levels of independent block operations, each
// block operation done by one thread in registers), and the FP32 solution is refined with
// residuals computed in double-float arithmetic (48-bit significand) until the correction
// falls below 2^-47 of the iterate, which brings the result to FP64-level accuracy.  Native
// FP64 is avoided: on this part it runs at about 1/60 of the FP32 rate with a 64-cycle
// dependent latency.  The factor storage lives in shared memory when it fits, else in global
// memory (L2 resident).
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
  float inv_omega_in, inv_omega_end;
};
__device__ __forceinline__ float kc_inv_omega(const KCompressed& k, int i) {
  return (i == 0 || i == k.n - 1) ? k.inv_omega_end : k.inv_omega_in;
}

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

// ---------------------------------------------------------------- register block kernels
template <int B>
__device__ __forceinline__ void blk_load(float (&a)[B * B], const float* p) {
#pragma unroll
  for (int i = 0; i < B * B; ++i) a[i] = p[i];
}
template <int B>
__device__ __forceinline__ void blk_store(float* p, const float (&a)[B * B]) {
#pragma unroll
  for (int i = 0; i < B * B; ++i) p[i] = a[i];
}
// In-place Cholesky L L^T of a row-major block: strict lower triangle holds L, the diagonal
// holds 1 / L_jj (reciprocal pivots, so the triangular solves only multiply).  False on a
// non-positive pivot.
template <int B>
__device__ __forceinline__ bool blk_chol(float (&a)[B * B]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    float d = a[j * B + j];
#pragma unroll
    for (int k = 0; k < j; ++k) d -= a[j * B + k] * a[j * B + k];
    if (!(d > 0.f)) { ok = false; d = 1.f; }
    const float inv = rsqrtf(d);
    a[j * B + j] = inv;
#pragma unroll
    for (int i = j + 1; i < B; ++i) {
      float v = a[i * B + j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= a[i * B + k] * a[j * B + k];
      a[i * B + j] = v * inv;
    }
  }
  return ok;
}
// x <- (L L^T)^-1 x with the factor of blk_chol
template <int B>
__device__ __forceinline__ void blk_chol_solve(const float (&L)[B * B], float (&x)[B]) {
#pragma unroll
  for (int i = 0; i < B; ++i) {
    float v = x[i];
#pragma unroll
    for (int k = 0; k < i; ++k) v -= L[i * B + k] * x[k];
    x[i] = v * L[i * B + i];
  }
#pragma unroll
  for (int i = B - 1; i >= 0; --i) {
    float v = x[i];
#pragma unroll
    for (int k = i + 1; k < B; ++k) v -= L[k * B + i] * x[k];
    x[i] = v * L[i * B + i];
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
template <int B>
__device__ inline bool cr_factor_t(const CRBuffers& s) {
  constexpr int BB = B * B;
  int ok = 1;
  int st = 1, K = s.nb;
  while (K > 1) {
    const int nodd = K / 2, neven = (K + 1) / 2;
    // odd blocks: Cholesky of D_j, G1 = D_j^-1 E[j-st], G2 = D_j^-1 E[j]^T
    for (int q = threadIdx.x; q < nodd; q += blockDim.x) {
      const int k = 2 * q + 1, j = k * st;
      float L[BB];
      blk_load<B>(L, s.D + j * BB);
      if (!blk_chol<B>(L)) ok = 0;
      blk_store<B>(s.D + j * BB, L);
      float e[BB], g[BB];
      blk_load<B>(e, s.E + (j - st) * BB);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float x[B];
#pragma unroll
        for (int r = 0; r < B; ++r) x[r] = e[r * B + c];
        blk_chol_solve<B>(L, x);
#pragma unroll
        for (int r = 0; r < B; ++r) g[r * B + c] = x[r];
      }
      blk_store<B>(s.G1 + j * BB, g);
      if (k + 1 < K) {
        blk_load<B>(e, s.E + j * BB);
#pragma unroll
        for (int c = 0; c < B; ++c) {
          float x[B];
#pragma unroll
          for (int r = 0; r < B; ++r) x[r] = e[c * B + r];
          blk_chol_solve<B>(L, x);
#pragma unroll
          for (int r = 0; r < B; ++r) g[r * B + c] = x[r];
        }
      } else {
#pragma unroll
        for (int i = 0; i < BB; ++i) g[i] = 0.f;
      }
      blk_store<B>(s.G2 + j * BB, g);
    }
    __syncthreads();
    // even blocks: Schur updates of D_i and the new coupling E[i] (i <-> i + 2st)
    for (int q = threadIdx.x; q < neven; q += blockDim.x) {
      const int k = 2 * q, i = k * st;
      float d[BB];
      blk_load<B>(d, s.D + i * BB);
      if (k >= 1) {                                  // E[j] G2[j], j = i - st
        const int j = i - st;
        float e[BB], g[BB];
        blk_load<B>(e, s.E + j * BB);
        blk_load<B>(g, s.G2 + j * BB);
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int c = 0; c < B; ++c) {
            float acc = d[r * B + c];
#pragma unroll
            for (int l = 0; l < B; ++l) acc -= e[r * B + l] * g[l * B + c];
            d[r * B + c] = acc;
          }
      }
      if (k + 1 < K) {                               // E[i]^T G1[j], j = i + st
        const int j = i + st;
        float e[BB], g[BB];
        blk_load<B>(e, s.E + i * BB);
        blk_load<B>(g, s.G1 + j * BB);
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int c = 0; c < B; ++c) {
            float acc = d[r * B + c];
#pragma unroll
            for (int l = 0; l < B; ++l) acc -= e[l * B + r] * g[l * B + c];
            d[r * B + c] = acc;
          }
        if (k + 2 < K) {                             // E[i] <- -E[j] G1[j]
          float e2[BB], n2[BB];
          blk_load<B>(e2, s.E + j * BB);
#pragma unroll
          for (int r = 0; r < B; ++r)
#pragma unroll
            for (int c = 0; c < B; ++c) {
              float acc = 0.f;
#pragma unroll
              for (int l = 0; l < B; ++l) acc -= e2[r * B + l] * g[l * B + c];
              n2[r * B + c] = acc;
            }
          blk_store<B>(s.E + i * BB, n2);
        }
      }
      blk_store<B>(s.D + i * BB, d);
    }
    __syncthreads();
    st *= 2;
    K = (K + 1) / 2;
  }
  if (threadIdx.x == 0) {
    float L[BB];
    blk_load<B>(L, s.D);
    if (!blk_chol<B>(L)) ok = 0;
    blk_store<B>(s.D, L);
  }
  return __syncthreads_and(ok) != 0;
}

// Solve with the factors; right-hand side in s.F (nb*b, padded rows zero), result in s.X.
template <int B>
__device__ inline void cr_solve_t(const CRBuffers& s) {
  constexpr int BB = B * B;
  int st = 1, K = s.nb, levels = 0;
  while (K > 1) {
    const int nodd = K / 2;
    // one task per active block: odd -> y_j = D_j^-1 f_j ; even -> f_i update
    for (int q = threadIdx.x; q < K; q += blockDim.x) {
      const int i = q * st;
      if (q & 1) {
        float L[BB], x[B];
        blk_load<B>(L, s.D + i * BB);
#pragma unroll
        for (int r = 0; r < B; ++r) x[r] = s.F[i * B + r];
        blk_chol_solve<B>(L, x);
#pragma unroll
        for (int r = 0; r < B; ++r) s.Y[i * B + r] = x[r];
      } else {
        float f[B];
#pragma unroll
        for (int r = 0; r < B; ++r) f[r] = s.F[i * B + r];
        if (q >= 1) {                                // - G2[j]^T f_j, j = i - st
          const int j = i - st;
          float g[BB], fj[B];
          blk_load<B>(g, s.G2 + j * BB);
#pragma unroll
          for (int l = 0; l < B; ++l) fj[l] = s.F[j * B + l];
#pragma unroll
          for (int r = 0; r < B; ++r)
#pragma unroll
            for (int l = 0; l < B; ++l) f[r] -= g[l * B + r] * fj[l];
        }
        if (q + 1 < K) {                             // - G1[j]^T f_j, j = i + st
          const int j = i + st;
          float g[BB], fj[B];
          blk_load<B>(g, s.G1 + j * BB);
#pragma unroll
          for (int l = 0; l < B; ++l) fj[l] = s.F[j * B + l];
#pragma unroll
          for (int r = 0; r < B; ++r)
#pragma unroll
            for (int l = 0; l < B; ++l) f[r] -= g[l * B + r] * fj[l];
        }
        // stage in Y (the odd F values are still being read this level)
#pragma unroll
        for (int r = 0; r < B; ++r) s.Y[i * B + r] = f[r];
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < K; q += blockDim.x) {
      if (q & 1) continue;
      const int i = q * st;
#pragma unroll
      for (int r = 0; r < B; ++r) s.F[i * B + r] = s.Y[i * B + r];
    }
    __syncthreads();
    (void)nodd;
    st *= 2;
    K = (K + 1) / 2;
    ++levels;
  }
  if (threadIdx.x == 0) {
    float L[BB], x[B];
    blk_load<B>(L, s.D);
#pragma unroll
    for (int r = 0; r < B; ++r) x[r] = s.F[r];
    blk_chol_solve<B>(L, x);
#pragma unroll
    for (int r = 0; r < B; ++r) s.X[r] = x[r];
  }
  __syncthreads();
  for (int lv = levels - 1; lv >= 0; --lv) {
    st = 1 << lv;
    K = (s.nb + st - 1) / st;
    const int nodd = K / 2;
    for (int q = threadIdx.x; q < nodd; q += blockDim.x) {
      const int k = 2 * q + 1, j = k * st;
      float x[B], xl[B], g[BB];
#pragma unroll
      for (int r = 0; r < B; ++r) { x[r] = s.Y[j * B + r]; xl[r] = s.X[(j - st) * B + r]; }
      blk_load<B>(g, s.G1 + j * BB);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int l = 0; l < B; ++l) x[r] -= g[r * B + l] * xl[l];
      if (k + 1 < K) {
        float xr[B];
#pragma unroll
        for (int r = 0; r < B; ++r) xr[r] = s.X[(j + st) * B + r];
        blk_load<B>(g, s.G2 + j * BB);
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int l = 0; l < B; ++l) x[r] -= g[r * B + l] * xr[l];
      }
#pragma unroll
      for (int r = 0; r < B; ++r) s.X[j * B + r] = x[r];
    }
    __syncthreads();
  }
}

static __device__ __noinline__ bool cr_factor(const CRBuffers& s) {
  switch (s.b) {
    case 3: return cr_factor_t<3>(s);
    case 5: return cr_factor_t<5>(s);
    default: return cr_factor_t<7>(s);
  }
}
static __device__ __noinline__ void cr_solve(const CRBuffers& s) {
  switch (s.b) {
    case 3: cr_solve_t<3>(s); break;
    case 5: cr_solve_t<5>(s); break;
    default: cr_solve_t<7>(s); break;
  }
}

// ---------------------------------------------------------------- first level on the fly
// For systems whose full factor storage exceeds shared memory: the odd blocks of level 0 are
// eliminated with their ORIGINAL blocks, rebuilt from the compressed band whenever needed (so
// they are never stored); the even blocks form the half-size level-1 system, which is
// factorised by cr_factor in shared memory.  With A_II the diagonal blocks and E_I the
// coupling of block I+1 to block I, for even i = 2q:
//   D1[q] = A_ii - E_{i-1} A_{i-1,i-1}^-1 E_{i-1}^T - E_i^T A_{i+1,i+1}^-1 E_i
//   E1[q] = -E_{i+1} A_{i+1,i+1}^-1 E_i             (coupling of level-1 blocks q+1 and q)
struct L0Buffers {
  float *F, *Y0, *X;    // full-length vectors (nb * b), global memory
  int nb, b;
  CRBuffers l1;         // level-1 system (ceil(nb/2) blocks)
};

template <int B>
__device__ __forceinline__ void band_diag_block(const KCompressed& k, int I, float a1, float a2, float (&d)[B * B]) {
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const int row = I * B + r, col = I * B + c;
      float v;
      if (row < k.n && col < k.n) {
        v = a2 * kc_entry(k, row, col - row).x;
        if (r == c) v += a1 * kc_omega(k, row).x;
      } else {
        v = (r == c) ? 1.f : 0.f;
      }
      d[r * B + c] = v;
    }
}
// E_I: rows of block I+1, columns of block I (zero past the end)
template <int B>
__device__ __forceinline__ void band_coupling_block(const KCompressed& k, int I, int nb, float a2, float (&e)[B * B]) {
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const int row = (I + 1) * B + r, col = I * B + c;
      float v = 0.f;
      if (I + 1 < nb && row < k.n && col < k.n && row - col <= B) v = a2 * kc_entry(k, row, col - row).x;
      e[r * B + c] = v;
    }
}

template <int B>
__device__ inline bool l0_factor_t(const L0Buffers& s, const KCompressed& k, float a1, float a2) {
  constexpr int BB = B * B;
  const int nb = s.nb, nb1 = s.l1.nb;
  for (int q = threadIdx.x; q < nb1; q += blockDim.x) {
    const int i = 2 * q;
    float d[BB], e1[BB];
    band_diag_block<B>(k, i, a1, a2, d);
#pragma unroll
    for (int t = 0; t < BB; ++t) e1[t] = 0.f;
    if (i >= 1) {                       // - E_{i-1} A_jj^-1 E_{i-1}^T, j = i - 1
      float L[BB], e[BB];
      band_diag_block<B>(k, i - 1, a1, a2, L);
      blk_chol<B>(L);
      band_coupling_block<B>(k, i - 1, nb, a2, e);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float x[B];
#pragma unroll
        for (int r = 0; r < B; ++r) x[r] = e[c * B + r];      // column c of E^T = row c of E
        blk_chol_solve<B>(L, x);                               // column c of A_jj^-1 E^T
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int l = 0; l < B; ++l) d[r * B + c] -= e[r * B + l] * x[l];
      }
    }
    if (i + 1 < nb) {                   // - E_i^T A_j'j'^-1 E_i, j' = i + 1; new coupling
      float L[BB], e[BB], e3[BB], g[BB];
      band_diag_block<B>(k, i + 1, a1, a2, L);
      blk_chol<B>(L);
      band_coupling_block<B>(k, i, nb, a2, e);
#pragma unroll
      for (int c = 0; c < B; ++c) {
        float x[B];
#pragma unroll
        for (int r = 0; r < B; ++r) x[r] = e[r * B + c];      // column c of E_i
        blk_chol_solve<B>(L, x);
#pragma unroll
        for (int r = 0; r < B; ++r) g[r * B + c] = x[r];      // G = A_j'j'^-1 E_i
      }
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) {
          float acc = d[r * B + c];
#pragma unroll
          for (int l = 0; l < B; ++l) acc -= e[l * B + r] * g[l * B + c];
          d[r * B + c] = acc;
        }
      if (i + 2 < nb) {
        band_coupling_block<B>(k, i + 1, nb, a2, e3);
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int c = 0; c < B; ++c) {
            float acc = 0.f;
#pragma unroll
            for (int l = 0; l < B; ++l) acc -= e3[r * B + l] * g[l * B + c];
            e1[r * B + c] = acc;
          }
      }
    }
    blk_store<B>(s.l1.D + q * BB, d);
    blk_store<B>(s.l1.E + q * BB, e1);
  }
  __syncthreads();
  return cr_factor_t<B>(s.l1);
}

// Solve with right-hand side s.F (nb*b, padded rows zero); result in s.X.
template <int B>
__device__ inline void l0_solve_t(const L0Buffers& s, const KCompressed& k, float a1, float a2) {
  constexpr int BB = B * B;
  const int nb = s.nb, nb1 = s.l1.nb;
  for (int q = threadIdx.x; 2 * q + 1 < nb; q += blockDim.x) {      // y_j = A_jj^-1 f_j, j odd
    const int j = 2 * q + 1;
    float L[BB], x[B];
    band_diag_block<B>(k, j, a1, a2, L);
    blk_chol<B>(L);
#pragma unroll
    for (int r = 0; r < B; ++r) x[r] = s.F[j * B + r];
    blk_chol_solve<B>(L, x);
#pragma unroll
    for (int r = 0; r < B; ++r) s.Y0[j * B + r] = x[r];
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nb1; q += blockDim.x) {             // level-1 right-hand side
    const int i = 2 * q;
    float f[B];
#pragma unroll
    for (int r = 0; r < B; ++r) f[r] = s.F[i * B + r];
    if (i >= 1) {                                                    // - E_{i-1} y_{i-1}
      float e[BB];
      band_coupling_block<B>(k, i - 1, nb, a2, e);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int l = 0; l < B; ++l) f[r] -= e[r * B + l] * s.Y0[(i - 1) * B + l];
    }
    if (i + 1 < nb) {                                                // - E_i^T y_{i+1}
      float e[BB];
      band_coupling_block<B>(k, i, nb, a2, e);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int l = 0; l < B; ++l) f[r] -= e[l * B + r] * s.Y0[(i + 1) * B + l];
    }
#pragma unroll
    for (int r = 0; r < B; ++r) s.l1.F[q * B + r] = f[r];
  }
  __syncthreads();
  cr_solve_t<B>(s.l1);
  for (int t = threadIdx.x; t < nb1 * B; t += blockDim.x) {
    const int q = t / B, r = t - q * B;
    s.X[2 * q * B + r] = s.l1.X[t];
  }
  __syncthreads();
  for (int q = threadIdx.x; 2 * q + 1 < nb; q += blockDim.x) {      // odd blocks back
    const int j = 2 * q + 1;
    float t[B], e[BB], L[BB];
#pragma unroll
    for (int r = 0; r < B; ++r) t[r] = 0.f;
    band_coupling_block<B>(k, j - 1, nb, a2, e);                      // E_{j-1} x_{j-1}
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int l = 0; l < B; ++l) t[r] += e[r * B + l] * s.X[(j - 1) * B + l];
    if (j + 1 < nb) {                                                 // E_j^T x_{j+1}
      band_coupling_block<B>(k, j, nb, a2, e);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int l = 0; l < B; ++l) t[r] += e[l * B + r] * s.X[(j + 1) * B + l];
    }
    band_diag_block<B>(k, j, a1, a2, L);
    blk_chol<B>(L);
    blk_chol_solve<B>(L, t);
#pragma unroll
    for (int r = 0; r < B; ++r) s.X[j * B + r] = s.Y0[j * B + r] - t[r];
  }
  __syncthreads();
}

static __device__ __noinline__ bool l0_factor(const L0Buffers& s, const KCompressed& k, float a1, float a2) {
  switch (s.b) {
    case 3: return l0_factor_t<3>(s, k, a1, a2);
    case 5: return l0_factor_t<5>(s, k, a1, a2);
    default: return l0_factor_t<7>(s, k, a1, a2);
  }
}
static __device__ __noinline__ void l0_solve(const L0Buffers& s, const KCompressed& k, float a1, float a2) {
  switch (s.b) {
    case 3: l0_solve_t<3>(s, k, a1, a2); break;
    case 5: l0_solve_t<5>(s, k, a1, a2); break;
    default: l0_solve_t<7>(s, k, a1, a2); break;
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

// ---------------------------------------------------------------- Chebyshev inner solver
// The D-scaled operator D^-1 (a1 D + a2 K) has its spectrum in [a1, a1 + a2 mu_max] exactly:
// K is positive semi-definite with the constants as null space (Neumann) and mu_max bounds the
// largest generalised eigenvalue of (K, D) (Gershgorin bound computed on the host).  The
// Chebyshev semi-iteration with these bounds needs no inner products: every iteration is one
// banded product and two vector updates over all rows in parallel, one __syncthreads.
struct ChebBuffers {
  float *r, *e, *d0, *d1;   // [n] residual, accumulated solution, two search vectors
  float* kb;                // explicit band rows near the two ends, FP32 ([nlead + ntail][2b+1], <= 256)
  float *F, *X;             // aliases used by the refinement loop (F = r, X = e)
};

__host__ __device__ inline int cheb_iterations(float a1, float a2, float mu_max, float tau) {
  const float kappa = (a1 + a2 * mu_max) / a1;
  const float sk = sqrtf(kappa);
  const float rho = (sk - 1.f) / (sk + 1.f);
  if (!(rho > 1e-30f)) return 1;
  const int k = static_cast<int>(ceilf(logf(2.f / tau) / logf(1.f / rho))) + 1;
  return k < 1 ? 1 : k;
}

// e = A^-1 r approximately (Chebyshev semi-iteration with D scaling), r overwritten.  The band
// descriptor is copied into registers and the interior stencil held in registers: the vectors
// live in shared memory and their stores would otherwise force descriptor reloads.
// Register-resident Chebyshev.  Threads 0 .. blockDim.x-33 own the interior rows in contiguous
// runs of R (R odd, so a warp's strided shared-memory accesses hit 32 different banks); the
// last warp's lanes own the explicit end rows (lane l < nlead: row l; lane 16 + l: row
// n - ntail + l).  Residual, iterate and search direction stay in registers; each iteration
// publishes the search direction to shared memory once (alternating buffers, zero padded by B
// on both sides) and reads back only the neighbours it needs.
template <int B, int R>
__device__ inline void cheb_solve_reg(const ChebBuffers& s, const KCompressed& kref, float a1, float a2, int iters,
                                      float theta, float delta, float sigma) {
  const KCompressed k = kref;
  const int n = k.n;
  constexpr int W = 2 * B + 1;
  float st[W];
#pragma unroll
  for (int o = 0; o < W; ++o) st[o] = a2 * k.stencil[o].x;
  const int ilo = k.nlead, ihi = n - k.ntail;
  const int tint = blockDim.x - 32;                 // interior threads
  const bool endlane = threadIdx.x >= tint;
  const int lane = threadIdx.x - tint;
  int i0 = 0, cnt = 0;                              // interior run [i0, i0 + cnt)
  int ie = -1;                                      // end row of an end lane
  if (!endlane) {
    i0 = ilo + threadIdx.x * R;
    cnt = max(0, min(R, ihi - i0));
  } else if (lane < k.nlead) {
    ie = lane;
  } else if (lane >= 16 && lane - 16 < k.ntail) {
    ie = n - k.ntail + (lane - 16);
  }
  // end rows: full band row (a2 K) in shared memory
  const int nx = k.nlead + k.ntail;
  for (int t = threadIdx.x; t < nx * W; t += blockDim.x) s.kb[t] = a2 * k.rows[t].x;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    s.d0[i] = 0.f; s.d0[n + B + i] = 0.f;
    s.d1[i] = 0.f; s.d1[n + B + i] = 0.f;
  }
  const float a1in = a1 * k.omega_in.x, iwin = k.inv_omega_in;
  float r[R], e[R], d[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    r[j] = j < cnt ? s.r[i0 + j] : 0.f;
    e[j] = 0.f;
    d[j] = r[j] * iwin / theta;
  }
  float re = 0.f, ee = 0.f, de = 0.f, iwe = 0.f, a1e = 0.f;
  const float* kre = nullptr;
  if (ie >= 0) {
    iwe = kc_inv_omega(k, ie);
    a1e = a1 * kc_omega(k, ie).x;
    re = s.r[ie];
    de = re * iwe / theta;
    kre = s.kb + (ie < ilo ? ie : k.nlead + ie - ihi) * W;
  }
  float rho_old = 1.f / sigma;
  for (int it = 0; it < iters; ++it) {
    float* dsh = ((it & 1) ? s.d1 : s.d0) + B;
    if (!endlane) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (j < cnt) dsh[i0 + j] = d[j];
    } else if (ie >= 0) {
      dsh[ie] = de;
    }
    __syncthreads();
    const float rho = 1.f / (2.f * sigma - rho_old);
    const float c1 = rho * rho_old, c2 = 2.f * rho / delta;
    if (!endlane) {
      if (cnt > 0) {
        // window rows i0 - B .. i0 + R + B - 1; own rows from registers, the rest from the
        // published vector (rows >= n read the zero padding, rows past it are zero)
        float win[R + 2 * B];
#pragma unroll
        for (int t = 0; t < B; ++t) {
          win[t] = dsh[i0 - B + t];
          const int row = i0 + R + t;
          win[R + B + t] = row < n + B ? dsh[row] : 0.f;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int row = i0 + j;
          win[B + j] = j < cnt ? d[j] : (row < n + B ? dsh[row] : 0.f);
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          float acc = a1in * d[j];
#pragma unroll
          for (int o = 0; o < W; ++o) acc = __fmaf_rn(st[o], win[j + o], acc);
          e[j] += d[j];
          r[j] -= acc;
          d[j] = __fmaf_rn(c1, d[j], c2 * (r[j] * iwin));
        }
      }
    } else if (ie >= 0) {
      float acc = a1e * de;
#pragma unroll
      for (int o = 0; o < W; ++o) acc = __fmaf_rn(kre[o], dsh[ie + o - B], acc);
      ee += de;
      re -= acc;
      de = __fmaf_rn(c1, de, c2 * (re * iwe));
    }
    rho_old = rho;
  }
  if (!endlane) {
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (j < cnt) s.e[i0 + j] = e[j];
  } else if (ie >= 0) {
    s.e[ie] = ee;
  }
  __syncthreads();
}

template <int B>
__device__ inline void cheb_solve_b(const ChebBuffers& s, const KCompressed& k, float a1, float a2, int iters,
                                    float theta, float delta, float sigma) {
  const int tint = blockDim.x - 32;
  const int nint = k.n - k.nlead - k.ntail;
  const int need = (nint + tint - 1) / tint;
  if (need <= 1) cheb_solve_reg<B, 1>(s, k, a1, a2, iters, theta, delta, sigma);
  else if (need <= 3) cheb_solve_reg<B, 3>(s, k, a1, a2, iters, theta, delta, sigma);
  else if (need <= 5) cheb_solve_reg<B, 5>(s, k, a1, a2, iters, theta, delta, sigma);
  else if (need <= 11) cheb_solve_reg<B, 11>(s, k, a1, a2, iters, theta, delta, sigma);
  else cheb_solve_reg<B, 19>(s, k, a1, a2, iters, theta, delta, sigma);
}

static __device__ __noinline__ void cheb_solve(const ChebBuffers& s, const KCompressed& k, float a1, float a2,
                                               int iters, float theta, float delta, float sigma) {
  switch (k.b) {
    case 3: cheb_solve_b<3>(s, k, a1, a2, iters, theta, delta, sigma); break;
    case 5: cheb_solve_b<5>(s, k, a1, a2, iters, theta, delta, sigma); break;
    default: cheb_solve_b<7>(s, k, a1, a2, iters, theta, delta, sigma); break;
  }
}

// r = q - (a1 omega x + a2 K x) in double-float; returns max |r.hi| over this thread's rows
template <int B>
__device__ inline void residual_df_t(const KCompressed& kref, dfloat a1, dfloat a2, const float2* q, const float2* x,
                                     float* out, int npad) {
  const KCompressed k = kref;
  const int n = k.n;
  float2 st[2 * B + 1];
#pragma unroll
  for (int o = 0; o < 2 * B + 1; ++o) st[o] = k.stencil[o];
  const int ilo = k.nlead, ihi = n - k.ntail;
  for (int i = threadIdx.x; i < npad; i += blockDim.x) {
    if (i >= n) { out[i] = 0.f; continue; }
    dfloat kx = {0.f, 0.f};
    if (i >= ilo && i < ihi) {
#pragma unroll
      for (int o = 0; o < 2 * B + 1; ++o) {
        const float2 xj = x[i + o - B];
        kx = df_add(kx, df_mul(dfloat{st[o].x, st[o].y}, dfloat{xj.x, xj.y}));
      }
    } else {
      const int j0 = max(0, i - B), j1 = min(n - 1, i + B);
      for (int j = j0; j <= j1; ++j) {
        const float2 kij = kc_entry(k, i, j - i);
        const float2 xj = x[j];
        kx = df_add(kx, df_mul(dfloat{kij.x, kij.y}, dfloat{xj.x, xj.y}));
      }
    }
    const float2 om = kc_omega(k, i);
    const float2 xi = x[i];
    const dfloat ax = df_add(df_mul(a2, kx), df_mul(a1, df_mul(dfloat{om.x, om.y}, dfloat{xi.x, xi.y})));
    const dfloat rr = df_add(dfloat{q[i].x, q[i].y}, df_neg(ax));
    out[i] = rr.hi + rr.lo;
  }
}
static __device__ __noinline__ void residual_df(const KCompressed& k, dfloat a1, dfloat a2, const float2* q,
                                                const float2* x, float* out, int npad) {
  switch (k.b) {
    case 3: residual_df_t<3>(k, a1, a2, q, x, out, npad); break;
    case 5: residual_df_t<5>(k, a1, a2, q, x, out, npad); break;
    default: residual_df_t<7>(k, a1, a2, q, x, out, npad); break;
  }
}

// Solver storage: full block cyclic reduction (cr) or first level on the fly (l0).
struct SolverStore {
  int mode;           // 0: full CR factors in `cr`; 1: level-0 on the fly, level-1 factors in l0.l1;
                      // 3: Chebyshev semi-iteration (`ch`)
  CRBuffers cr;
  L0Buffers l0;
  ChebBuffers ch;
  float mu_max;       // Chebyshev: bound of the largest generalised eigenvalue of (K, D)
  float *F, *X;       // full-length right-hand side / solution of one pass
};

// Full solve with refinement.  q: double-float right-hand side [n]; x: double-float result
// [n].  a1, a2 as double-float.  Returns false on a failed pivot or a non-finite result.
static __device__ __noinline__ bool banded_solve(const SolverStore& s, const KCompressed& k, dfloat a1, dfloat a2,
                                    const float2* q, float2* x, float* red, unsigned long long* trace = nullptr,
                                    const float2* x0 = nullptr) {
  const int n = k.n, b = k.b;
  const int npad = s.mode == 3 ? n : (s.mode == 0 ? s.cr.nb : s.l0.nb) * b;
  unsigned long long t0 = trace ? global_ns() : 0ull;
  bool ok = true;
  int cheb_its = 0;
  float th = 0.f, de = 0.f, sg = 0.f;
  if (s.mode == 0) {
    cr_build(s.cr, k, a1.hi, a2.hi);
    __syncthreads();
    ok = cr_factor(s.cr);
  } else if (s.mode == 1) {
    ok = l0_factor(s.l0, k, a1.hi, a2.hi);
  } else {
    const float lmin = a1.hi, lmax = a1.hi + a2.hi * s.mu_max;
    th = 0.5f * (lmax + lmin);
    de = 0.5f * (lmax - lmin);
    if (!(de > 0.f)) de = 1e-30f * th;
    sg = th / de;
    cheb_its = cheb_iterations(a1.hi, a2.hi, s.mu_max, 2.384185791015625e-07f);   // 2^-22
    ok = (lmin > 0.f) && cheb_its < 100000;
    if (cheb_its > 4096) cheb_its = 4096;
  }
  if (trace && threadIdx.x == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveFactor, t - t0); t0 = t; }
  // per-pass contraction of the error: the Chebyshev bound 2^-22, or FP32 rounding times cond
  const float kappa = s.mode == 3 ? (a1.hi + a2.hi * s.mu_max) / a1.hi : 1.f;
  const float rho_pass = 4.f * fmaxf(2.384185791015625e-07f, kappa * 5.960464477539063e-08f);
  bool warm = x0 != nullptr && s.mode == 3;
  if (warm) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = x0[i];
    __syncthreads();
  } else {
    for (int i = threadIdx.x; i < npad; i += blockDim.x) s.F[i] = (i < n) ? q[i].x : 0.f;
    __syncthreads();
    if (s.mode == 0) cr_solve(s.cr);
    else if (s.mode == 1) l0_solve(s.l0, k, a1.hi, a2.hi);
    else cheb_solve(s.ch, k, a1.hi, a2.hi, cheb_its, th, de, sg);
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = make_float2(s.X[i], 0.f);
    __syncthreads();
  }
  if (trace && threadIdx.x == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveFirst, t - t0); t0 = t; }
  float prev = 0.f;
  for (int it = 0; it < 4; ++it) {
    // r = q - (a1 omega x + a2 K x) in double-float
    residual_df(k, a1, a2, q, x, s.F, npad);
    __syncthreads();
    if (s.mode == 0) cr_solve(s.cr);
    else if (s.mode == 1) l0_solve(s.l0, k, a1.hi, a2.hi);
    else cheb_solve(s.ch, k, a1.hi, a2.hi, cheb_its, th, de, sg);
    float dmax = 0.f, xmax = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const dfloat nx = df_add(dfloat{x[i].x, x[i].y}, dfloat{s.X[i], 0.f});
      x[i] = make_float2(nx.hi, nx.lo);
      dmax = fmaxf(dmax, fabsf(s.X[i]));
      xmax = fmaxf(xmax, fabsf(nx.hi));
    }
    dmax = cta_max(dmax, red);
    xmax = cta_max(xmax, red);
    if (trace && threadIdx.x == 0) atomicAdd(trace + kTrSolvePasses, 1ull);
    if (!(dmax == dmax) || !(xmax <= 3.0e38f)) return false;   // NaN / Inf
    // the refinement contracts the error by rho ~ dmax / prev per pass; stop once the next
    // correction would fall below 2^-48 of the iterate (or this one already did)
    if (dmax <= 3.552713678800501e-15f * xmax) break;
    if (s.mode == 3 && rho_pass * dmax <= 3.552713678800501e-15f * xmax) break;
    if (it > 0 && prev > 0.f && dmax * (dmax / prev) <= 3.552713678800501e-15f * xmax) break;
    prev = dmax;
  }
  if (trace && threadIdx.x == 0) atomicAdd(trace + kTrSolveRefine, global_ns() - t0);
  return ok;
}

// Shared / global floats each solver mode needs for n rows of half bandwidth b.
__host__ __device__ inline size_t l0_smem_floats(int n, int b) {
  const int nb = (n + b - 1) / b, nb1 = (nb + 1) / 2;
  return cr_floats(nb1 * b, b);
}
__host__ __device__ inline size_t l0_global_floats(int n, int b) {
  const int nb = (n + b - 1) / b;
  return static_cast<size_t>(nb) * b * 3;
}

__host__ __device__ inline size_t cheb_floats(int n) { return static_cast<size_t>(n) * 4 + 32 + 256; }

// Bind solver storage.  mode 0: factors at fbase; mode 1: level-1 factors at fbase, full vectors
// at gbase; mode 3: Chebyshev vectors at fbase.
__device__ inline SolverStore solver_bind(int mode, float* fbase, float* gbase, int n, int b, float mu_max = 0.f) {
  SolverStore s;
  s.mode = mode;
  s.mu_max = mu_max;
  if (mode == 3) {
    s.ch.r = fbase;
    s.ch.e = fbase + n;
    s.ch.d0 = fbase + 2 * n;            // n + 2B published search direction (B <= 7)
    s.ch.d1 = fbase + 3 * n + 16;
    s.ch.kb = fbase + 4 * n + 32;
    s.ch.F = s.ch.r;
    s.ch.X = s.ch.e;
    s.F = s.ch.r;
    s.X = s.ch.e;
  } else if (mode == 0) {
    s.cr = cr_bind(fbase, n, b);
    s.F = s.cr.F;
    s.X = s.cr.X;
  } else {
    const int nb = (n + b - 1) / b, nb1 = (nb + 1) / 2;
    s.l0.nb = nb;
    s.l0.b = b;
    s.l0.F = gbase;
    s.l0.Y0 = gbase + nb * b;
    s.l0.X = gbase + 2 * nb * b;
    s.l0.l1 = cr_bind(fbase, nb1 * b, b);
    s.F = s.l0.F;
    s.X = s.l0.X;
  }
  return s;
}

}  // namespace ctd

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
  // Consistent mass of the Gauss rule in the same compressed form (null: the nodal rule's
  // diagonal mass diag(omega))
  int mlead, mtail;
  const float2* mrows;
  const float2* mstencil;
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
// Mass entry M[i][i + off]: the consistent band (Gauss rule) or diag(omega) (nodal rule)
__device__ __forceinline__ float2 kc_mass(const KCompressed& k, int i, int off /* -b..b */) {
  if (!k.mrows) return off == 0 ? kc_omega(k, i) : make_float2(0.f, 0.f);
  const int w = 2 * k.b + 1;
  if (i < k.mlead) return k.mrows[i * w + off + k.b];
  if (i >= k.n - k.mtail) return k.mrows[(k.mlead + i - (k.n - k.mtail)) * w + off + k.b];
  return k.mstencil[off + k.b];
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
    if (row < n && col < n && (row - col <= b && col - row <= b)) {
      dv = a2 * kc_entry(k, row, col - row).x;
      if (k.mrows) dv += a1 * kc_mass(k, row, col - row).x;
      else if (row == col) dv += a1 * kc_omega(k, row).x;
    } else {
      dv = (r == c) ? 1.f : 0.f;
      if (row < n && col < n) dv = 0.f;
    }
    s.D[t] = dv;
    const int row2 = row + b;
    float ev = 0.f;
    if (I + 1 < s.nb && row2 < n && col < n && row2 - col <= b) {
      ev = a2 * kc_entry(k, row2, col - row2).x;
      if (k.mrows) ev += a1 * kc_mass(k, row2, col - row2).x;
    }
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
        if (k.mrows) v += a1 * kc_mass(k, row, col - row).x;
        else if (r == c) v += a1 * kc_omega(k, row).x;
      } else {
        v = (r == c) ? 1.f : 0.f;
      }
      d[r * B + c] = v;
    }
}
// E_I: rows of block I+1, columns of block I (zero past the end)
template <int B>
__device__ __forceinline__ void band_coupling_block(const KCompressed& k, int I, int nb, float a1, float a2,
                                                    float (&e)[B * B]) {
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const int row = (I + 1) * B + r, col = I * B + c;
      float v = 0.f;
      if (I + 1 < nb && row < k.n && col < k.n && row - col <= B) {
        v = a2 * kc_entry(k, row, col - row).x;
        if (k.mrows) v += a1 * kc_mass(k, row, col - row).x;
      }
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
      band_coupling_block<B>(k, i - 1, nb, a1, a2, e);
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
      band_coupling_block<B>(k, i, nb, a1, a2, e);
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
        band_coupling_block<B>(k, i + 1, nb, a1, a2, e3);
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
      band_coupling_block<B>(k, i - 1, nb, a1, a2, e);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int l = 0; l < B; ++l) f[r] -= e[r * B + l] * s.Y0[(i - 1) * B + l];
    }
    if (i + 1 < nb) {                                                // - E_i^T y_{i+1}
      float e[BB];
      band_coupling_block<B>(k, i, nb, a1, a2, e);
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
    band_coupling_block<B>(k, j - 1, nb, a1, a2, e);                      // E_{j-1} x_{j-1}
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int l = 0; l < B; ++l) t[r] += e[r * B + l] * s.X[(j - 1) * B + l];
    if (j + 1 < nb) {                                                 // E_j^T x_{j+1}
      band_coupling_block<B>(k, j, nb, a1, a2, e);
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

// ---------------------------------------------------------------- Chebyshev solver
// The D-scaled operator D^-1 (a1 D + a2 K), D = diag(omega), has its spectrum in
// [a1, a1 + a2 mu_max] exactly: K is positive semi-definite (the constants span its null space
// under the Neumann boundary) and mu_max bounds the largest generalised eigenvalue of (K, D)
// (Gershgorin bound computed on the host).  The Chebyshev semi-iteration with these bounds
// needs no inner products: an iteration is one banded product and three vector updates.
//
// Work split of the CTA (T = blockDim.x threads, tint = T - 32):
//  * interior thread t < tact owns the R consecutive rows nlead + t R .. nlead + (t + 1) R - 1
//    (uniform stencil, uniform nodal weight);
//  * the last warp owns the end rows: the nlead explicit rows at the start and the rows
//    [e0, n) at the end (the explicit tail rows and the interior rows left over), at most
//    kChebEndMax, two per lane;
//  * residual, correction and search direction stay in registers.  Each iteration a thread
//    publishes only what its neighbours read (an interior thread its first and last B values,
//    an end lane its rows) into one of two alternating buffers, meets the others at one
//    __syncthreads and reads its halo back.  Interior rows go in pairs through the packed
//    FP32x2 instructions of sm_100 and later.
// Each pass solves for the correction of a double-float residual; passes repeat until the
// remaining error is bounded by 2^-46 of the iterate.
struct ChebLayout {
  int nl;      // lead rows of the end warp: the explicit ones, plus one so that interior rows
               // start at an even index (row pairs are 16-byte aligned in shared memory)
  int R;       // rows per interior thread
  int tint;    // interior threads (blockDim.x - 32)
  int tact;    // interior threads that own rows
  int e0;      // first row of the end region at the tail
  int nend;    // rows of the end warp
};
constexpr int kChebEndMax = 64;
constexpr int kChebRowOptions = 4;
constexpr int kChebRegion = 80;   // publication slots of one end region (rows -B .. +B around it)

__host__ __device__ inline int cheb_rows_option(int q) {
  switch (q) {
    case 0: return 4;
    case 1: return 8;
    case 2: return 12;
    default: return 20;
  }
}

// Smallest R (> b, so that halos come from the immediate neighbours) whose split leaves at
// most kChebEndMax end rows.  False if none does.
__host__ __device__ inline bool cheb_layout(int n, int nlead, int ntail, int b, int tint, ChebLayout& L) {
  int nl = nlead + (nlead & 1);
  if (nl + ntail > n) nl = nlead;
  const int nint = n - nl - ntail;
  if (nint < 0) return false;
  for (int q = 0; q < kChebRowOptions; ++q) {
    const int R = cheb_rows_option(q);
    if (R <= b) continue;
    int tact = nint / R;
    if (tact > tint) tact = tint;
    const int nend = nl + ntail + (nint - tact * R);
    if (nend > kChebEndMax) continue;
    if (tact > 0 && (nl < b + 1 || ntail < b || (nl & 1))) return false;   // halos, alignment
    L.nl = nl;
    L.R = R;
    L.tint = tint;
    L.tact = tact;
    L.e0 = nl + tact * R;
    L.nend = nend;
    return true;
  }
  return false;
}

// Floats of one publication buffer: Hl [b][tint] (first b values of each interior thread),
// Hr [b][tint] (last b values), then the lead and tail regions in natural row order with b
// slots of zeros or interior values on either side (kChebRegion each), then four slots that
// threads without rows write and nobody reads.
__host__ __device__ inline int cheb_buffer_floats(int b, int tint) { return 2 * b * tint + 2 * kChebRegion + 4; }

struct ChebSmem {
  float2* q;     // [n] right-hand side staged from global memory (double-float)
  float2* kbd;   // [kChebEndMax][2b+1] K rows of the end rows (double-float)
  float2* st;    // [2b+1] interior stencil of K (double-float)
  float* halo;   // [2][S] publication buffers
  float* kb;     // [kChebEndMax][2b+1] a2 K + a1 omega rows of the end rows (FP32)
  float* rs;     // [n] residual / correction of the interior rows (FP32)
  float* red;    // [64] reduction scratch
  int S;         // floats per publication buffer
};

__host__ __device__ inline size_t cheb_floats(int n) {
  return static_cast<size_t>((n + 3) & ~3) * 3 + static_cast<size_t>(kChebEndMax) * 15 * 3 + 32 +
         2 * static_cast<size_t>(cheb_buffer_floats(7, 256 - 32)) + 64;
}

__host__ __device__ inline int cheb_iterations(float a1, float a2, float mu_max, float tau) {
  const float kappa = (a1 + a2 * mu_max) / a1;
  const float sk = sqrtf(kappa);
  const float rho = (sk - 1.f) / (sk + 1.f);
  if (!(rho > 1e-30f)) return 1;
  const int k = static_cast<int>(ceilf(logf(2.f / tau) / logf(1.f / rho))) + 1;
  return k < 1 ? 1 : k;
}

__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}

// s + c += a * x for double-float a, x: the high products are summed with an error-free
// transformation (TwoSum, plus the FMA residual of each product) into the FP32 compensation c.
__device__ __forceinline__ void df_dot_acc(float& s, float& c, float2 a, float2 x) {
  const float p = a.x * x.x;
  const float pe = __fmaf_rn(a.x, x.x, -p);
  const float t = s + p;
  const float bb = t - s;
  const float se = (s - (t - bb)) + (p - bb);
  s = t;
  c += se + pe;
  c = __fmaf_rn(a.x, x.y, c);
  c = __fmaf_rn(a.y, x.x, c);
}

// q_i - (a1 omega_i x_i + a2 (K x)_i) rounded to FP32, from the row's 2B+1 products (s, c).
__device__ __forceinline__ float df_residual_finish(float s, float c, dfloat a1w, dfloat a2, float2 xi, float2 qi) {
  const dfloat kx = df_two_sum(s, c);
  const dfloat ax = df_add(df_mul(a2, kx), df_mul(a1w, dfloat{xi.x, xi.y}));
  const dfloat rr = df_add(dfloat{qi.x, qi.y}, df_neg(ax));
  return rr.hi + rr.lo;
}

// ---- two double-float values side by side (rows i, i + 1), FP32x2 instructions; the same
// operation order as the scalar dfloat routines, so the results are identical.
struct df2 { float2 hi, lo; };
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ df2 df2_two_sum(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 bb = f2_sub(s, a);
  const float2 e = __fadd2_rn(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
  return {s, e};
}
__device__ __forceinline__ df2 df2_fast_two_sum(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return {s, f2_sub(b, f2_sub(s, a))};
}
__device__ __forceinline__ df2 df2_add(df2 a, df2 b) {
  df2 s = df2_two_sum(a.hi, b.hi);
  const df2 t = df2_two_sum(a.lo, b.lo);
  s.lo = __fadd2_rn(s.lo, t.hi);
  s = df2_fast_two_sum(s.hi, s.lo);
  s.lo = __fadd2_rn(s.lo, t.lo);
  return df2_fast_two_sum(s.hi, s.lo);
}
// a * b for a double-float scalar a
__device__ __forceinline__ df2 df2_mul_s(dfloat a, df2 b) {
  const float2 ah = make_float2(a.hi, a.hi), al = make_float2(a.lo, a.lo);
  const float2 p = __fmul2_rn(ah, b.hi);
  float2 e = __ffma2_rn(ah, b.hi, make_float2(-p.x, -p.y));
  e = __ffma2_rn(ah, b.lo, e);
  e = __ffma2_rn(al, b.hi, e);
  return df2_fast_two_sum(p, e);
}
// df_dot_acc for two rows at once: s + c += a * x
__device__ __forceinline__ void df2_dot_acc(float2& s, float2& c, float2 a, float2 xh, float2 xl) {
  const float2 ah = make_float2(a.x, a.x), al = make_float2(a.y, a.y);
  const float2 p = __fmul2_rn(ah, xh);
  const float2 pe = __ffma2_rn(ah, xh, make_float2(-p.x, -p.y));
  const float2 t = __fadd2_rn(s, p);
  const float2 bb = f2_sub(t, s);
  const float2 se = __fadd2_rn(f2_sub(s, f2_sub(t, bb)), f2_sub(p, bb));
  s = t;
  c = __fadd2_rn(c, __fadd2_rn(se, pe));
  c = __ffma2_rn(ah, xl, c);
  c = __ffma2_rn(al, xh, c);
}

__device__ __forceinline__ void bar_sync_all() { asm volatile("bar.sync 0;" ::: "memory"); }

// 8-byte global -> shared copy that bypasses registers; completed by cp_async_wait_all.
__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem))),
               "l"(src_gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Error bound of one pass of `its` Chebyshev iterations (x4 margin), FP32 rounding included.
__device__ __forceinline__ float cheb_pass_bound(float rho, int its, float kappa) {
  const float cheb = 2.f * exp2f(static_cast<float>(its) * log2f(rho));
  return 4.f * fmaxf(cheb, kappa * 5.960464477539063e-08f);
}

// Relative accuracy a solve stops at: 2^-48 of the iterate (the double-float limit) for the
// FP64 path; 2^-34 for the tensor-core path, whose contraction carries FP32 rounding into
// every right-hand side (2^-34 is 5.8e-11, far below that).
constexpr float kSolveTolFp64 = 3.552713678800501e-15f;
constexpr float kSolveTolMixed = 5.820766091346741e-11f;
// Error reduction of a first refinement pass: 2^-22, unless the caller knows its warm start
// to be closer (then tol over the expected relative change, at most 2^-8)
constexpr float kFirstPassTau = 2.384185791015625e-07f;

// End of a refinement pass, executed by every thread: CTA max of the correction and of the
// iterate, trace, and the decision: 0 next pass (with `its` iterations), 1 converged, -1
// non-finite values.  The error left after the pass is at most bound * dmax; the pass stops
// the solve once that is below tol of the iterate, else the next pass gets just enough
// iterations to get there (never fewer than the FP32 rounding floor allows).
__device__ __forceinline__ int cheb_pass_end(float dmax, float xmax, float& bound, int& its, int pass, float a1,
                                             float a2, float mu_max, float rho, float kappa, float* red,
                                             unsigned long long* trace, unsigned long long& tsub, float tol) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  }
  const int tid = threadIdx.x;
  if ((tid & 31) == 0) { red[tid >> 5] = dmax; red[32 + (tid >> 5)] = xmax; }
  bar_sync_all();
  dmax = 0.f;
  xmax = 0.f;
  for (int q = 0; q < static_cast<int>(blockDim.x >> 5); ++q) { dmax = fmaxf(dmax, red[q]); xmax = fmaxf(xmax, red[32 + q]); }
  bar_sync_all();
  if (trace && tid == 0) {
    atomicAdd(trace + kTrSolvePasses, 1ull);
    const unsigned long long t = global_ns();
    atomicAdd(trace + (pass == 0 ? kTrSolveFirst : kTrSolveRefine), t - tsub);
    tsub = t;
  }
  if (!(dmax <= 3.0e38f) || !(xmax <= 3.0e38f)) return -1;
  const float lim = tol * xmax;
  if (dmax <= lim || bound * dmax <= lim) return 1;
  const float need = lim / (2.f * bound * dmax);      // reduction the next pass must reach
  const float floor32 = 4.f * kappa * 5.960464477539063e-08f;
  const float tau = need > floor32 ? fminf(need, 0.5f) : 2.384185791015625e-07f;
  its = cheb_iterations(a1, a2, mu_max, tau);
  if (its > 4096) its = 4096;
  bound = cheb_pass_bound(rho, its, kappa);
  return 0;
}

// Interior threads: `its` Chebyshev iterations on their R rows.  Threads without rows run the
// same code on zeros with dummy slots, so that every warp of the interior group executes the
// same barrier instructions.  nst: -(a1 omega + a2 K) stencil, packed.
template <int B, int R>
__device__ __forceinline__ void cheb_iterate_interior(float (&r)[R], float (&e)[R], float (&w)[R + 2 * B + 2],
                                                      const float2 (&nst)[2 * B + 1], float iwin, int its,
                                                      float sigma, float inv2d, uint32_t pub_l, uint32_t spl,
                                                      uint32_t pub_r, uint32_t spr, uint32_t src_l, uint32_t str_l,
                                                      uint32_t src_r, uint32_t str_r, uint32_t bufb) {
  constexpr int W = 2 * B + 1;
  constexpr int OWN = B + 1;
  float rho_old = 1.f / sigma;
  for (int it = 0; it < its; ++it) {
    const uint32_t boff = (it & 1) ? bufb : 0u;
#pragma unroll
    for (int q = 0; q < B; ++q) {
      sts_f32(pub_l + boff + q * spl, w[OWN + q]);
      sts_f32(pub_r + boff + q * spr, w[OWN + R - B + q]);
    }
    bar_sync_all();
    const float rho = __fdividef(1.f, 2.f * sigma - rho_old);
    const float c1 = rho * rho_old, c2 = rho * inv2d * iwin;
#pragma unroll
    for (int q = 0; q < B; ++q) {
      w[1 + q] = lds_f32(src_l + boff + q * str_l);
      w[R + B + 1 + q] = lds_f32(src_r + boff + q * str_r);
    }
#pragma unroll
    for (int m = 0; m < R / 2; ++m) {
      float2 acc = make_float2(r[2 * m], r[2 * m + 1]);
      // symmetric stencil: the pair sums d_{j-B+o} + d_{j+B-o} go through the adder, leaving
      // B + 1 multiply-adds per row pair
      acc = __ffma2_rn(nst[B], make_float2(w[2 * m + 1 + B], w[2 * m + 2 + B]), acc);
#pragma unroll
      for (int o = 0; o < B; ++o) {
        const float2 sum = __fadd2_rn(make_float2(w[2 * m + 1 + o], w[2 * m + 2 + o]),
                                      make_float2(w[2 * m + 1 + 2 * B - o], w[2 * m + 2 + 2 * B - o]));
        acc = __ffma2_rn(nst[o], sum, acc);
      }
      r[2 * m] = acc.x;
      r[2 * m + 1] = acc.y;
    }
    const float2 c1v = make_float2(c1, c1), c2v = make_float2(c2, c2);
#pragma unroll
    for (int m = 0; m < R / 2; ++m) {
      const float2 dd = make_float2(w[OWN + 2 * m], w[OWN + 2 * m + 1]);
      const float2 ev = __fadd2_rn(make_float2(e[2 * m], e[2 * m + 1]), dd);
      e[2 * m] = ev.x;
      e[2 * m + 1] = ev.y;
      const float2 nd = __ffma2_rn(c1v, dd, __fmul2_rn(c2v, make_float2(r[2 * m], r[2 * m + 1])));
      w[OWN + 2 * m] = nd.x;
      w[OWN + 2 * m + 1] = nd.y;
    }
    rho_old = rho;
  }
}

// End lanes: `its` Chebyshev iterations on up to two explicit rows each (row coefficients in
// shared memory, a1 omega folded into the diagonal).
template <int B>
__device__ __forceinline__ void cheb_iterate_end(float (&er)[2], float (&ee)[2], float (&ed)[2], const int (&erow)[2],
                                                 const uint32_t (&epub)[2], const uint32_t (&ewin)[2],
                                                 const uint32_t (&ekb)[2], const float (&eiw)[2], int its,
                                                 float sigma, float inv2d, uint32_t bufb) {
  constexpr int W = 2 * B + 1;
  float rho_old = 1.f / sigma;
  for (int it = 0; it < its; ++it) {
    const uint32_t boff = (it & 1) ? bufb : 0u;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
      if (erow[s2] >= 0) sts_f32(epub[s2] + boff, ed[s2]);
    bar_sync_all();
    const float rho = __fdividef(1.f, 2.f * sigma - rho_old);
    const float c1 = rho * rho_old, c2 = rho * inv2d;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      if (erow[s2] < 0) continue;
      float acc = 0.f;
#pragma unroll
      for (int o = 0; o < W; ++o)
        acc = __fmaf_rn(lds_f32(ekb[s2] + 4u * o), o == B ? ed[s2] : lds_f32(ewin[s2] + boff + 4u * o), acc);
      ee[s2] += ed[s2];
      er[s2] -= acc;
      ed[s2] = __fmaf_rn(c1, ed[s2], c2 * (er[s2] * eiw[s2]));
    }
    rho_old = rho;
  }
}

template <int B, int R>
__device__ bool cheb_solve_t(const KCompressed& kref, const ChebLayout& Lref, dfloat a1, dfloat a2, float mu_max,
                             const float2* qg, float2* x, const float2* x0, const ChebSmem& smref,
                             unsigned long long* trace, float tol, float tau0) {
  constexpr int W = 2 * B + 1;
  constexpr int NW = R + 2 * B + 2;   // window: halo rows at [1, B + 1) and [R + B + 1, R + 2B + 1)
  constexpr int OWN = B + 1;          // own row j at w[OWN + j] (even index: rows pair up)
  const KCompressed k = kref;
  const ChebLayout L = Lref;
  const ChebSmem sm = smref;
  const int n = k.n, tid = threadIdx.x, T = blockDim.x;
  unsigned long long tsub = trace ? global_ns() : 0ull;

  // ---- Chebyshev constants (FP32 is enough for the iteration count)
  const float lmin = a1.hi, lmax = a1.hi + a2.hi * mu_max;
  const float theta = 0.5f * (lmax + lmin);
  float delta = 0.5f * (lmax - lmin);
  if (!(delta > 0.f)) delta = 1e-30f * theta;
  const float sigma = theta / delta, inv2d = 2.f / delta, c0 = 1.f / theta;
  const float kappa = lmax / lmin;
  const float sk = sqrtf(kappa), crho = (sk - 1.f) / (sk + 1.f);
  int its = cheb_iterations(a1.hi, a2.hi, mu_max, tau0);   // first pass: error reduction tau0
  const bool ok = (lmin > 0.f) && its < 100000;
  if (its > 4096) its = 4096;
  float bound = cheb_pass_bound(crho, its, kappa);

  // ---- stage q, the warm start, the stencil and the end rows (double-float) with async copies
  const int reg0 = 2 * B * L.tint;               // lead region: slot B + row
  const int reg1 = reg0 + kChebRegion;           // tail region: slot B + row - e0 (tact > 0)
  const int trash = reg1 + kChebRegion;          // written by threads without rows, never read
  const bool warm = x0 != nullptr;
  for (int i = tid; i < n; i += T) {
    cp_async8(sm.q + i, qg + i);
    if (warm) cp_async8(x + i, x0 + i);
  }
  if (tid < W) cp_async8(sm.st + tid, k.stencil + tid);
  for (int c = tid; c < L.nend * W; c += T) {
    const int slot = c / W, o = c - slot * W;
    const int row = slot < L.nl ? slot : L.e0 + (slot - L.nl);
    const float2* src = row < k.nlead ? k.rows + row * W + o
                        : row >= n - k.ntail ? k.rows + (k.nlead + row - (n - k.ntail)) * W + o
                                             : k.stencil + o;
    cp_async8(sm.kbd + c, src);
  }
  for (int c = tid; c < 4 * kChebRegion; c += T)
    sm.halo[(c / (2 * kChebRegion)) * sm.S + reg0 + c % (2 * kChebRegion)] = 0.f;
  cp_async_wait_all();
  __syncthreads();
  // FP32 operator rows of the end rows: a2 K + a1 omega on the diagonal, zero outside [0, n)
  for (int c = tid; c < L.nend * W; c += T) {
    const int slot = c / W, o = c - slot * W;
    const int row = slot < L.nl ? slot : L.e0 + (slot - L.nl);
    const int j = row + o - B;
    float v = (j >= 0 && j < n) ? a2.hi * sm.kbd[c].x : 0.f;
    if (o == B) v += a1.hi * kc_omega(k, row).x;
    sm.kb[c] = v;
  }
  __syncthreads();

  const uint32_t hbase = static_cast<uint32_t>(__cvta_generic_to_shared(sm.halo));
  const uint32_t bufb = 4u * static_cast<uint32_t>(sm.S);
  if (trace && tid == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveFactor, t - tsub); tsub = t; }
  bool fail = false;

  if (tid < L.tint) {
    // ================= interior group
    const bool active = tid < L.tact;
    const int i0 = L.nl + tid * R;
    const int npairs = (L.e0 - L.nl) / 2;   // interior row pairs
    const uint32_t kstr = 4u * static_cast<uint32_t>(L.tint);
    const float a1in = a1.hi * k.omega_in.x, iwin = k.inv_omega_in;
    // -(a1 omega + a2 K) stencil in FP32, symmetrised (K is symmetric; this operator only
    // drives the inner iterations, the residual uses the stored double-float stencil)
    float2 nst[W];
#pragma unroll
    for (int o = 0; o < W; ++o) {
      const int om = W - 1 - o;
      const float v = o == B ? -(a2.hi * sm.st[o].x + a1in) : -(a2.hi * 0.5f * (sm.st[o].x + sm.st[om].x));
      nst[o] = make_float2(v, v);
    }
    const dfloat a1w_in = df_mul(a1, dfloat{k.omega_in.x, k.omega_in.y});
    // where the first / last B values are published and the halos read; the outer interior
    // threads use the end regions, threads without rows a trash slot and the zero slots
    uint32_t pub_l = hbase + 4u * trash, pub_r = hbase + 4u * trash, spl = 0u, spr = 0u;
    uint32_t src_l = hbase + 4u * reg0, src_r = hbase + 4u * reg0, str_l = 0u, str_r = 0u;
    if (active) {
      if (tid == 0) {
        pub_l = hbase + 4u * (reg0 + B + L.nl);             // rows nl .. nl + B - 1
        spl = 4u;
        src_l = hbase + 4u * (reg0 + L.nl);                 // rows nl - B .. nl - 1
        str_l = 4u;
      } else {
        pub_l = hbase + 4u * tid;
        spl = kstr;
        src_l = hbase + 4u * (B * L.tint + tid - 1);
        str_l = kstr;
      }
      if (tid == L.tact - 1) {
        pub_r = hbase + 4u * reg1;                          // rows e0 - B .. e0 - 1
        spr = 4u;
        src_r = hbase + 4u * (reg1 + B);                    // rows e0 .. e0 + B - 1
        str_r = 4u;
      } else {
        pub_r = hbase + 4u * (B * L.tint + tid);
        spr = kstr;
        src_r = hbase + 4u * (tid + 1);
        str_r = kstr;
      }
    }
    float r[R], e[R], w[NW];
    for (int pass = 0; pass < 6; ++pass) {
      const bool cold0 = !warm && pass == 0;
      unsigned long long tp = trace ? global_ns() : 0ull;
      // Residual of the current iterate (double-float), rounded to FP32, into sm.rs[row - nl].
      // Here consecutive threads take consecutive row pairs (16-byte aligned): conflict-free
      // shared-memory accesses; the loop stays rolled (unrolled, it is tens of KB of code
      // fetched anew on every pass).
      if (cold0) {
#pragma unroll 1
        for (int p = tid; p < npairs; p += L.tint) {
          const int i = L.nl + 2 * p;
          const float4 qq = *reinterpret_cast<const float4*>(sm.q + i);
          *reinterpret_cast<float2*>(sm.rs + 2 * p) = make_float2(qq.x + qq.y, qq.z + qq.w);
        }
      } else {
        float2 sdf[W];
#pragma unroll
        for (int o = 0; o < W; ++o) sdf[o] = sm.st[o];
#pragma unroll 1
        for (int p = tid; p < npairs; p += L.tint) {
          const int i = L.nl + 2 * p;
          float2 xw[2 * B + 4];   // rows i - B - 1 .. i + B + 2
#pragma unroll
          for (int c = 0; c < B + 2; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(x + i - B - 1 + 2 * c);
            xw[2 * c] = make_float2(v.x, v.y);
            xw[2 * c + 1] = make_float2(v.z, v.w);
          }
          const float4 qq = *reinterpret_cast<const float4*>(sm.q + i);
          float2 s2 = make_float2(0.f, 0.f), c2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int o = 0; o < W; ++o) {
            const float2 xa = xw[o + 1], xb = xw[o + 2];
            df2_dot_acc(s2, c2, sdf[o], make_float2(xa.x, xb.x), make_float2(xa.y, xb.y));
          }
          const float2 x0v = xw[B + 1], x1v = xw[B + 2];
          const df2 kx = df2_two_sum(s2, c2);
          const df2 ax = df2_add(df2_mul_s(a2, kx),
                                 df2_mul_s(a1w_in, df2{make_float2(x0v.x, x1v.x), make_float2(x0v.y, x1v.y)}));
          const df2 rr = df2_add(df2{make_float2(qq.x, qq.z), make_float2(qq.y, qq.w)},
                                 df2{make_float2(-ax.hi.x, -ax.hi.y), make_float2(-ax.lo.x, -ax.lo.y)});
          *reinterpret_cast<float2*>(sm.rs + 2 * p) = __fadd2_rn(rr.hi, rr.lo);
        }
      }
      bar_sync_all();
      if (trace && tid == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveResidual, t - tp); tp = t; }
      // own rows of this thread (R consecutive, 16-byte aligned in sm.rs)
#pragma unroll
      for (int j = 0; j < R; j += 4) {
        const float4 v = active ? *reinterpret_cast<const float4*>(sm.rs + tid * R + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        r[j] = v.x;
        r[j + 1] = v.y;
        r[j + 2] = v.z;
        r[j + 3] = v.w;
      }
#pragma unroll
      for (int j = 0; j < NW; ++j) w[j] = 0.f;
#pragma unroll
      for (int j = 0; j < R; ++j) { e[j] = 0.f; w[OWN + j] = r[j] * iwin * c0; }
      cheb_iterate_interior<B, R>(r, e, w, nst, iwin, its, sigma, inv2d, pub_l, spl, pub_r, spr, src_l, str_l, src_r,
                                  str_r, bufb);
      if (trace && tid == 0) atomicAdd(trace + kTrSolveInner, global_ns() - tp);
      // x += e (double-float) over row pairs, size of the correction and of the iterate.  The
      // iterations' last barrier orders every read of sm.rs above before these writes.
      if (active) {
#pragma unroll
        for (int j = 0; j < R; j += 4)
          *reinterpret_cast<float4*>(sm.rs + tid * R + j) = make_float4(e[j], e[j + 1], e[j + 2], e[j + 3]);
      }
      bar_sync_all();
      float dmax = 0.f, xmax = 0.f;
#pragma unroll 1
      for (int p = tid; p < npairs; p += L.tint) {
        const int i = L.nl + 2 * p;
        const float2 ev = *reinterpret_cast<const float2*>(sm.rs + 2 * p);
        const float4 xo = cold0 ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(x + i);
        const dfloat n0 = df_add(dfloat{xo.x, xo.y}, dfloat{ev.x, 0.f});
        const dfloat n1 = df_add(dfloat{xo.z, xo.w}, dfloat{ev.y, 0.f});
        *reinterpret_cast<float4*>(x + i) = make_float4(n0.hi, n0.lo, n1.hi, n1.lo);
        dmax = fmaxf(dmax, fmaxf(fabsf(ev.x), fabsf(ev.y)));
        xmax = fmaxf(xmax, fmaxf(fabsf(n0.hi), fabsf(n1.hi)));
        if (!(fabsf(ev.x) <= 3.0e38f) || !(fabsf(ev.y) <= 3.0e38f)) dmax = __int_as_float(0x7f800000);
      }
      const int stop = cheb_pass_end(dmax, xmax, bound, its, pass, a1.hi, a2.hi, mu_max, crho, kappa, sm.red, trace,
                                     tsub, tol);
      if (stop) { fail = stop < 0; break; }
    }
  } else {
    // ================= end warp
    const int lane = tid - L.tint;
    int erow[2] = {-1, -1};
    uint32_t epub[2] = {0u, 0u}, ewin[2] = {0u, 0u}, ekb[2] = {0u, 0u};
    int eslot[2] = {0, 0};
    float eiw[2] = {0.f, 0.f};
    dfloat ea1wd[2] = {{0.f, 0.f}, {0.f, 0.f}};
    const uint32_t kbase = static_cast<uint32_t>(__cvta_generic_to_shared(sm.kb));
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int slot = lane + 32 * s2;
      if (slot < L.nend) {
        const int row = slot < L.nl ? slot : L.e0 + (slot - L.nl);
        erow[s2] = row;
        eslot[s2] = slot;
        const float2 om = kc_omega(k, row);
        ea1wd[s2] = df_mul(a1, dfloat{om.x, om.y});
        eiw[s2] = kc_inv_omega(k, row);
        const int ps = (L.tact == 0 || row < L.nl) ? reg0 + B + row : reg1 + B + (row - L.e0);
        epub[s2] = hbase + 4u * ps;
        ewin[s2] = hbase + 4u * (ps - B);
        ekb[s2] = kbase + 4u * (slot * W);
      }
    }
    float er[2], ee[2], ed[2];
    for (int pass = 0; pass < 6; ++pass) {
      const bool cold0 = !warm && pass == 0;
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        er[s2] = 0.f;
        const int row = erow[s2];
        if (row < 0) continue;
        if (cold0) {
          const float2 qq = sm.q[row];
          er[s2] = qq.x + qq.y;
        } else {
          float s = 0.f, c = 0.f;
          const float2* kr = sm.kbd + eslot[s2] * W;
#pragma unroll
          for (int o = 0; o < W; ++o) {
            const int j = row + o - B;
            if (j >= 0 && j < n) df_dot_acc(s, c, kr[o], x[j]);
          }
          er[s2] = df_residual_finish(s, c, ea1wd[s2], a2, x[row], sm.q[row]);
        }
      }
      bar_sync_all();   // matches the interior group's barrier after its residual
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) { ee[s2] = 0.f; ed[s2] = er[s2] * eiw[s2] * c0; }
      cheb_iterate_end<B>(er, ee, ed, erow, epub, ewin, ekb, eiw, its, sigma, inv2d, bufb);
      bar_sync_all();   // matches the interior group's barrier before its update
      float dmax = 0.f, xmax = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2) {
        const int row = erow[s2];
        if (row < 0) continue;
        const float2 xo = cold0 ? make_float2(0.f, 0.f) : x[row];
        const dfloat nx = df_add(dfloat{xo.x, xo.y}, dfloat{ee[s2], 0.f});
        x[row] = make_float2(nx.hi, nx.lo);
        dmax = fmaxf(dmax, fabsf(ee[s2]));
        xmax = fmaxf(xmax, fabsf(nx.hi));
        if (!(fabsf(ee[s2]) <= 3.0e38f)) dmax = __int_as_float(0x7f800000);
      }
      const int stop = cheb_pass_end(dmax, xmax, bound, its, pass, a1.hi, a2.hi, mu_max, crho, kappa, sm.red, trace,
                                     tsub, tol);
      if (stop) { fail = stop < 0; break; }
    }
  }
  __syncthreads();
  return ok && !fail;
}

static __device__ __noinline__ bool cheb_banded_solve(const KCompressed& k, dfloat a1, dfloat a2, float mu_max,
                                                      const float2* q, float2* x, const float2* x0,
                                                      const ChebSmem& sm, unsigned long long* trace, float tol,
                                                      float tau0) {
  ChebLayout L;
  if (!cheb_layout(k.n, k.nlead, k.ntail, k.b, static_cast<int>(blockDim.x) - 32, L)) return false;
  switch (k.b * 100 + L.R) {
    case 304: return cheb_solve_t<3, 4>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 308: return cheb_solve_t<3, 8>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 312: return cheb_solve_t<3, 12>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 320: return cheb_solve_t<3, 20>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 508: return cheb_solve_t<5, 8>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 512: return cheb_solve_t<5, 12>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 520: return cheb_solve_t<5, 20>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 708: return cheb_solve_t<7, 8>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 712: return cheb_solve_t<7, 12>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    case 720: return cheb_solve_t<7, 20>(k, L, a1, a2, mu_max, q, x, x0, sm, trace, tol, tau0);
    default: return false;
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
    dfloat mx;
    if (k.mrows) {   // consistent mass (Gauss rule): band product
      mx = {0.f, 0.f};
      const int j0 = max(0, i - B), j1 = min(n - 1, i + B);
      for (int j = j0; j <= j1; ++j) {
        const float2 mij = kc_mass(k, i, j - i);
        const float2 xj = x[j];
        mx = df_add(mx, df_mul(dfloat{mij.x, mij.y}, dfloat{xj.x, xj.y}));
      }
    } else {
      const float2 om = kc_omega(k, i);
      const float2 xi = x[i];
      mx = df_mul(dfloat{om.x, om.y}, dfloat{xi.x, xi.y});
    }
    const dfloat ax = df_add(df_mul(a2, kx), df_mul(a1, mx));
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
  ChebSmem ch;
  float mu_max;       // Chebyshev: bound of the largest generalised eigenvalue of (K, D)
  float *F, *X;       // full-length right-hand side / solution of one pass
};

// Full solve with refinement.  q: double-float right-hand side [n]; x: double-float result
// [n].  a1, a2 as double-float.  Returns false on a failed pivot or a non-finite result.
static __device__ __noinline__ bool banded_solve(const SolverStore& s, const KCompressed& k, dfloat a1, dfloat a2,
                                    const float2* q, float2* x, float* red, unsigned long long* trace = nullptr,
                                    const float2* x0 = nullptr, float tol = kSolveTolFp64,
                                    float tau0 = kFirstPassTau) {
  if (s.mode == 3) return cheb_banded_solve(k, a1, a2, s.mu_max, q, x, x0, s.ch, trace, tol, tau0);
  const int n = k.n, b = k.b;
  const int npad = (s.mode == 0 ? s.cr.nb : s.l0.nb) * b;
  unsigned long long t0 = trace ? global_ns() : 0ull;
  bool ok = true;
  if (s.mode == 0) {
    cr_build(s.cr, k, a1.hi, a2.hi);
    __syncthreads();
    ok = cr_factor(s.cr);
  } else {
    ok = l0_factor(s.l0, k, a1.hi, a2.hi);
  }
  if (trace && threadIdx.x == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveFactor, t - t0); t0 = t; }
  for (int i = threadIdx.x; i < npad; i += blockDim.x) s.F[i] = (i < n) ? q[i].x : 0.f;
  __syncthreads();
  if (s.mode == 0) cr_solve(s.cr);
  else l0_solve(s.l0, k, a1.hi, a2.hi);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = make_float2(s.X[i], 0.f);
  __syncthreads();
  if (trace && threadIdx.x == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveFirst, t - t0); t0 = t; }
  float prev = 0.f;
  for (int it = 0; it < 4; ++it) {
    // r = q - (a1 omega x + a2 K x) in double-float
    unsigned long long tp = trace ? global_ns() : 0ull;
    residual_df(k, a1, a2, q, x, s.F, npad);
    __syncthreads();
    if (trace && threadIdx.x == 0) { const unsigned long long t = global_ns(); atomicAdd(trace + kTrSolveResidual, t - tp); tp = t; }
    if (s.mode == 0) cr_solve(s.cr);
    else l0_solve(s.l0, k, a1.hi, a2.hi);
    if (trace && threadIdx.x == 0) atomicAdd(trace + kTrSolveInner, global_ns() - tp);
    float dmax = 0.f, xmax = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const dfloat nx = df_add(dfloat{x[i].x, x[i].y}, dfloat{s.X[i], 0.f});
      x[i] = make_float2(nx.hi, nx.lo);
      dmax = fmaxf(dmax, fabsf(s.X[i]));
      if (!(fabsf(s.X[i]) <= 3.0e38f)) dmax = __int_as_float(0x7f800000);
      xmax = fmaxf(xmax, fabsf(nx.hi));
    }
    dmax = cta_max(dmax, red);
    xmax = cta_max(xmax, red);
    if (trace && threadIdx.x == 0) atomicAdd(trace + kTrSolvePasses, 1ull);
    if (!(dmax <= 3.0e38f) || !(xmax <= 3.0e38f)) return false;   // NaN / Inf
    // the refinement contracts the error by rho ~ dmax / prev per pass; stop once the next
    // correction would fall below 2^-48 of the iterate (or this one already did)
    if (dmax <= 3.552713678800501e-15f * xmax) break;
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

// Bind solver storage.  mode 0: factors at fbase; mode 1: level-1 factors at fbase, full vectors
// at gbase; mode 3: Chebyshev right-hand side, publication buffers and reduction scratch at fbase.
__device__ inline SolverStore solver_bind(int mode, float* fbase, float* gbase, int n, int b, float mu_max = 0.f) {
  SolverStore s;
  s.mode = mode;
  s.mu_max = mu_max;
  s.F = s.X = nullptr;
  if (mode == 3) {
    // q and rs are read as 16-byte vectors: both start on 16-byte boundaries (fbase is)
    const int n4 = (n + 3) & ~3;
    s.ch.q = reinterpret_cast<float2*>(fbase);
    s.ch.rs = fbase + 2 * n4;
    s.ch.kbd = reinterpret_cast<float2*>(s.ch.rs + n4);
    s.ch.st = s.ch.kbd + kChebEndMax * 15;
    s.ch.S = cheb_buffer_floats(b, static_cast<int>(blockDim.x) - 32);
    s.ch.halo = reinterpret_cast<float*>(s.ch.st + 16);
    s.ch.kb = s.ch.halo + 2 * s.ch.S;
    s.ch.red = s.ch.kb + kChebEndMax * 15;
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

// Device-side pieces of one CTD time step (Section 3.3) shared by the step kernel and the
// probe kernels: mode-bank access, Gram partial sums (the 1D products of Eq. KxQx),
// right-hand-side rows, the FP64 nonlinear contraction, convergence partials.
#pragma once
#include "ctd_common.cuh"
#include "ctd_solve.cuh"
#include "ctd_contract_tc.cuh"

namespace ctd {

// per other-dimension slot block of the Gram partials:
// [0] m = v^T M v, [1] k = v^T K v, [2, 2+Mcap) gM_j = v^T M b_j, [2+Mcap, 2+2Mcap) gK_j =
// v^T K b_j, [2+2Mcap, 2+3Mcap) h_j = v^T M a_j   (a_j: factors of u^k, b_j: of u^{k+1})
__host__ __device__ inline int slots_per_dim(int Mcap, int sep_q = 0) { return 2 + 3 * Mcap + sep_q; }

// Multisets {m1 <= m2 <= m3} in colex order (by m3, then m2, then m1), so that those with all
// indices below M_k are the first sep_terms(M_k); packed m1 | m2 << 8 | m3 << 16 | orderings << 24
// (orderings: 1, 3 or 6 ordered triples per multiset).
struct SepTable {
  unsigned e[kMaxSep];
};
constexpr SepTable make_sep_table() {
  SepTable t{};
  int q = 0;
  for (int m3 = 0; m3 < kMaxSepModes; ++m3)
    for (int m2 = 0; m2 <= m3; ++m2)
      for (int m1 = 0; m1 <= m2; ++m1) {
        const unsigned ord = (m1 == m3) ? 1u : ((m1 == m2 || m2 == m3) ? 3u : 6u);
        t.e[q++] = static_cast<unsigned>(m1) | (static_cast<unsigned>(m2) << 8) | (static_cast<unsigned>(m3) << 16) |
                   (ord << 24);
      }
  return t;
}
__constant__ SepTable kSepTable = make_sep_table();

// The separated form (Eq. MxySep) has its own translation unit and step kernel
// (ctd_kernels_sep.cu compiles ctd_kernels.cu with CTD_SEPARATED_TU); the grid form's kernel
// holds none of its code.  The separated form requires M_max <= kMaxSepModes, so every M_k is
// within the multiset table.
#ifdef CTD_SEPARATED_TU
constexpr bool kSepTU = true;
#else
constexpr bool kSepTU = false;
#endif
__device__ __forceinline__ bool sep_active(const StepParams&, int Mk) { return kSepTU && Mk > 0; }

struct Extra {            // per-launch workspace pieces not in StepParams
  KCompressed kc[kMaxDim];
  double* Af[kMaxDim];    // FP64 copy of u^k factors [Mcap][n] (FP64-path materialisation)
  double* maxpart;        // [kMaxDim][grid]
  int* ctrl;              // [4] solver flags broadcast
  double* rpart_tc;        // [nq][cmax] partial row sums of the tensor-core contraction (one per CTA)
  TcDir dirs[kMaxDim];    // tensor-core geometry per direction
  __nv_bfloat16* kr[kMaxDim];   // column operands per direction: 3D Khatri-Rao, cube form scaled
  int tc_stages;          // B-operand ring depth
  float2* xprev;          // [kMaxDim][kMaxN] last unnormalised solve per direction (warm start)
};

__device__ __forceinline__ dfloat ld_df(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void st_df(float2* p, dfloat v) { *p = make_float2(v.hi, v.lo); }
__device__ __forceinline__ dfloat df_of(double x) { return df_from_double(x); }

// K v at row i of dimension d (double-float), K read from the compressed band
__device__ inline dfloat kv_row(const KCompressed& k, const float2* v, int i) {
  constexpr int kW = 2 * 7 + 1;   // widest band (s = 3)
  float2 kv[kW], vv[kW];
#pragma unroll
  for (int o = 0; o < kW; ++o) {   // all loads first, so that their latencies overlap
    const int j = i + o - k.b;
    const bool ok = o <= 2 * k.b && j >= 0 && j < k.n;
    kv[o] = ok ? kc_entry(k, i, o - k.b) : make_float2(0.f, 0.f);
    vv[o] = ok ? v[j] : make_float2(0.f, 0.f);
  }
  dfloat acc = {0.f, 0.f};
#pragma unroll
  for (int o = 0; o < kW; ++o)
    if (o <= 2 * k.b) acc = df_fma(acc, dfloat{kv[o].x, kv[o].y}, dfloat{vv[o].x, vv[o].y});
  return acc;
}

// M v at row i of dimension d (double-float): the consistent mass band of the Gauss rule, or
// omega_i v_i under the nodal rule
__device__ inline dfloat mv_row(const KCompressed& k, const float2* v, int i) {
  if (!k.mrows) {
    const float2 om = kc_omega(k, i);
    return df_mul(dfloat{om.x, om.y}, ld_df(v + i));
  }
  constexpr int kW = 2 * 7 + 1;   // widest band (s = 3)
  float2 mv[kW], vv[kW];
#pragma unroll
  for (int o = 0; o < kW; ++o) {   // all loads first, so that their latencies overlap
    const int j = i + o - k.b;
    const bool ok = o <= 2 * k.b && j >= 0 && j < k.n;
    mv[o] = ok ? kc_mass(k, i, o - k.b) : make_float2(0.f, 0.f);
    vv[o] = ok ? v[j] : make_float2(0.f, 0.f);
  }
  dfloat acc = {0.f, 0.f};
#pragma unroll
  for (int o = 0; o < kW; ++o)
    if (o <= 2 * k.b) acc = df_fma(acc, dfloat{mv[o].x, mv[o].y}, dfloat{vv[o].x, vv[o].y});
  return acc;
}

// Value at Gauss point r of dimension d of the 1D function with nodal coefficients f
// (double-float): sum_k N~_{phi0[r]+k}(x_r) f[phi0[r]+k] (Gauss rule)
__device__ inline dfloat phi_row(const Dim& dd, int phiw, const float2* f, int r) {
  const int j0 = dd.phi0[r];
  const float2* ph = dd.phi + static_cast<size_t>(r) * kPhiW;
  dfloat acc = {0.f, 0.f};
  for (int k = 0; k < phiw; ++k) {
    const int j = j0 + k;
    if (j < dd.n) acc = df_fma(acc, ld_df(ph + k), ld_df(f + j));
  }
  return acc;
}

// Reduce a double-float value over the `tp` consecutive lanes of a group (tp power of 2 <=
// 32), fixed xor tree.
__device__ inline dfloat group_sum(dfloat v, int tp) {
  for (int o = tp >> 1; o > 0; o >>= 1) {
    dfloat u;
    u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, u);
  }
  return v;
}

__device__ inline int pow2_floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// ---------------------------------------------------------------------------------------
// Phase A (part 1): Gram partial sums for every dimension d != x over this CTA's slice of
// dimension d's nodes.  Writes gram[(o * spd + slot) * G + cta] for the used slots.
// Shared scratch: 3 * kChunk float2.
constexpr int kChunk = 256;
// Gram and convergence partial sums are computed by this many CTAs (fewer partials to reduce
// after the grid-wide wait: every CTA reads all of them)
constexpr int kGramCtas = kLightCtas;   // the lighter-loaded contraction CTAs

__device__ __forceinline__ int gram_ctas(const StepParams& P) { return P.vgrid < kGramCtas ? P.vgrid : kGramCtas; }

static __device__ __noinline__ void gram_partials(const StepParams& P, const Extra& X, int x, int Mk, int M,
                              int pb, int cb, float2* sh) {
  const int G = gram_ctas(P), cta = P.vrank, D = P.dim, spd = slots_per_dim(P.Mcap, P.sep_q);
  if (cta >= G) return;
  const int nsep = sep_active(P, Mk) ? sep_terms(Mk) : 0;
  float2* sv = sh;               // v_i
  float2* sdv = sh + kChunk;     // omega_i v_i
  float2* skv = sh + 2 * kChunk; // (K v)_i
  int o = 0;
  for (int d = 0; d < D; ++d) {
    if (d == x) continue;
    const Dim& dd = P.d[d];
    int lo, hi;
    slice_of(dd.n, G, cta, lo, hi);
    const int nbase = 2 + 2 * M + Mk;
    const int nslots = nbase + nsep;   // separated form: one slot per multiset
    // thread group per slot
    const int tp = min(32, pow2_floor(max(1, kThreads / max(1, nslots))));
    const int groups = kThreads / tp;
    const int g = threadIdx.x / tp, lane = threadIdx.x % tp;
    // accumulators for the (up to ceil(nslots/groups)) slots of this group
    dfloat acc[8];
    const int per = (nslots + groups - 1) / groups;   // <= 8 since nslots <= 2+5*128 ... guarded
    for (int k = 0; k < 8; ++k) acc[k] = {0.f, 0.f};
    for (int c0 = lo; c0 < hi; c0 += kChunk) {
      const int c1 = min(hi, c0 + kChunk);
      __syncthreads();
      for (int i = c0 + threadIdx.x; i < c1; i += kThreads) {
        const dfloat v = ld_df(dd.v + i);
        const float2 om = kc_omega(X.kc[d], i);
        st_df(sv + i - c0, v);
        st_df(sdv + i - c0, P.quad ? mv_row(X.kc[d], dd.v, i) : df_mul(dfloat{om.x, om.y}, v));
        st_df(skv + i - c0, kv_row(X.kc[d], dd.v, i));
      }
      __syncthreads();
      for (int k = 0; k < per; ++k) {
        const int s = g + k * groups;
        if (s >= nslots) break;
        dfloat a = acc[k];
        if (s >= nbase) {
          // separated form: sum_i (omega v)_i f_m1,i f_m2,i f_m3,i over factors of u^k
          const unsigned e = kSepTable.e[s - nbase];
          const float2* f1 = dd.bank[pb] + static_cast<size_t>(e & 0xFF) * dd.n + c0;
          const float2* f2 = dd.bank[pb] + static_cast<size_t>((e >> 8) & 0xFF) * dd.n + c0;
          const float2* f3 = dd.bank[pb] + static_cast<size_t>((e >> 16) & 0xFF) * dd.n + c0;
          for (int i = lane; i < c1 - c0; i += tp) {
            const float2 x1 = f1[i], x2 = f2[i], x3 = f3[i], w = sdv[i];
            const dfloat f = df_mul(df_mul(dfloat{x1.x, x1.y}, dfloat{x2.x, x2.y}), dfloat{x3.x, x3.y});
            a = df_fma(a, f, dfloat{w.x, w.y});
          }
          acc[k] = a;
          continue;
        }
        // the slot's two vectors: shared-memory staging (v, omega v, K v) or a factor column
        const float2 *lhs, *rhs;
        if (s == 0) { lhs = sv; rhs = sdv; }
        else if (s == 1) { lhs = sv; rhs = skv; }
        else if (s < 2 + M) { lhs = sdv; rhs = dd.bank[cb] + static_cast<size_t>(s - 2) * dd.n + c0; }
        else if (s < 2 + 2 * M) { lhs = sv; rhs = dd.KB + static_cast<size_t>(s - 2 - M) * dd.n + c0; }
        else { lhs = sdv; rhs = dd.bank[pb] + static_cast<size_t>(s - 2 - 2 * M) * dd.n + c0; }
        for (int i = lane; i < c1 - c0; i += 4 * tp) {
          float2 l4[4], r4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {   // four rows' loads first, so that their latencies overlap
            const int ii = i + u * tp;
            const bool ok = ii < c1 - c0;
            l4[u] = ok ? lhs[ii] : make_float2(0.f, 0.f);
            r4[u] = ok ? rhs[ii] : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) a = df_fma(a, dfloat{l4[u].x, l4[u].y}, dfloat{r4[u].x, r4[u].y});
        }
        acc[k] = a;
      }
    }
    for (int k = 0; k < per; ++k) {
      const int s = g + k * groups;
      const dfloat r = group_sum(acc[k], tp);   // all lanes of the warp participate
      if (s < nslots && lane == 0) {
        int slot;
        if (s < 2) slot = s;
        else if (s < 2 + M) slot = s;                               // gM
        else if (s < 2 + 2 * M) slot = 2 + P.Mcap + (s - 2 - M);    // gK
        else if (s < nbase) slot = 2 + 2 * P.Mcap + (s - 2 - 2 * M);  // h
        else slot = 2 + 3 * P.Mcap + (s - nbase);                   // separated multisets
        st_df(P.gram + static_cast<size_t>(o * spd + slot) * G + cta, r);
      }
    }
    ++o;
  }
}

// Coefficients of Eq. KxQx for direction x, in shared memory (double-float):
// coef[0] = alpha1, coef[1] = alpha2, H[m] = prod_{d!=x} h_d,m, GM[m] = prod gM_d,m,
// GK[m] = sum_{d'} gK_{d',m} prod_{d != x,d'} gM_d,m; separated form (Eq. MxySep):
// T[q] = orderings(q) prod_{d!=x} sum_i (omega v)_d,i f_m1 f_m2 f_m3 for multiset q.
struct Coef {
  float2 alpha1, alpha2;
  float2 H[kMaxModes], GM[kMaxModes], GK[kMaxModes];
  float2* T;   // [kMaxSep] in the phase's shared scratch, after the Gram sums
};

// Used Gram slots of one fixed dimension: m_d, k_d, gM (M), gK (M), h (Mk), separated (nsep)
__host__ __device__ inline int coef_slots(int M, int Mk, int nsep) { return 2 + 2 * M + Mk + nsep; }
constexpr size_t kCoefScratchSums = (kMaxDim - 1) * (2 + 3 * kMaxModes + kMaxSep);   // float2
constexpr size_t kCoefScratchBytes = sizeof(float2) * (kCoefScratchSums + kMaxSep);

// Every used slot's G partials are loaded at once (16 lanes per slot, lane g holds CTA g's
// partial, G <= 16) and summed by a fixed xor tree, so that all CTAs get the same bits.
// scratch: kCoefScratchBytes of shared memory.
static __device__ __noinline__ void build_coefficients(const StepParams& P, int x, int Mk, int M, Coef* c,
                                   float2* scratch) {
  const int G = gram_ctas(P), D = P.dim, spd = slots_per_dim(P.Mcap, P.sep_q);
  const int nsep = sep_active(P, Mk) ? sep_terms(Mk) : 0;
  const int nO = D - 1, per = coef_slots(M, Mk, nsep), nsl = nO * per;
  const int g = threadIdx.x & 15, sub = threadIdx.x >> 4;
  constexpr int kSub = kThreads / 16;   // slots per round
  constexpr int kRounds = 4;            // rounds whose loads are issued together
  for (int u0 = 0; u0 < nsl; u0 += kSub * kRounds) {
    float2 v[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int u = u0 + r * kSub + sub;
      v[r] = make_float2(0.f, 0.f);
      if (u < nsl && g < G) {
        const int o = u / per, k = u - o * per;
        int slot;
        if (k < 2 + M) slot = k;                                     // m_d, k_d, gM
        else if (k < 2 + 2 * M) slot = 2 + P.Mcap + (k - 2 - M);     // gK
        else if (k < 2 + 2 * M + Mk) slot = 2 + 2 * P.Mcap + (k - 2 - 2 * M);   // h
        else slot = 2 + 3 * P.Mcap + (k - 2 - 2 * M - Mk);           // separated multisets
        v[r] = P.gram[static_cast<size_t>(o * spd + slot) * G + g];
      }
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int u = u0 + r * kSub + sub;
      const dfloat t = group_sum(dfloat{v[r].x, v[r].y}, 16);
      if (u < nsl && g == 0) st_df(scratch + u, t);
    }
  }
  __syncthreads();
  for (int m = threadIdx.x; m < max(M, Mk); m += blockDim.x) {
    if (m < Mk) {
      dfloat H = {1.f, 0.f};
      for (int o = 0; o < nO; ++o) H = df_mul(H, ld_df(scratch + o * per + 2 + 2 * M + m));
      st_df(c->H + m, H);
    }
    if (m < M) {
      dfloat GM = {1.f, 0.f}, GK = {0.f, 0.f};
      for (int o = 0; o < nO; ++o) GM = df_mul(GM, ld_df(scratch + o * per + 2 + m));
      for (int o2 = 0; o2 < nO; ++o2) {
        dfloat t = ld_df(scratch + o2 * per + 2 + M + m);
        for (int o = 0; o < nO; ++o)
          if (o != o2) t = df_mul(t, ld_df(scratch + o * per + 2 + m));
        GK = df_add(GK, t);
      }
      st_df(c->GM + m, GM);
      st_df(c->GK + m, GK);
    }
  }
  if (threadIdx.x == 0) c->T = scratch + kCoefScratchSums;
  for (int q = threadIdx.x; q < nsep; q += blockDim.x) {
    dfloat t = {static_cast<float>(kSepTable.e[q] >> 24), 0.f};
    for (int o = 0; o < nO; ++o) t = df_mul(t, ld_df(scratch + o * per + 2 + 2 * M + Mk + q));
    st_df(scratch + kCoefScratchSums + q, t);
  }
  if (threadIdx.x == 0) {
    const dfloat ct = ld_df(&P.ct_df), ck = ld_df(&P.ck_df);
    dfloat pm = {1.f, 0.f}, stiff = {0.f, 0.f};
    for (int o = 0; o < nO; ++o) pm = df_mul(pm, ld_df(scratch + o * per));
    for (int o2 = 0; o2 < nO; ++o2) {
      dfloat t = ld_df(scratch + o2 * per + 1);
      for (int o = 0; o < nO; ++o)
        if (o != o2) t = df_mul(t, ld_df(scratch + o * per));
      stiff = df_add(stiff, t);
    }
    st_df(&c->alpha1, df_add(df_mul(ct, pm), df_mul(ck, stiff)));
    st_df(&c->alpha2, df_mul(ck, pm));
  }
  __syncthreads();
}

// Gauss rule: Phi_x^T of the point sums of the nonlinear contraction at node i, i.e. the sum
// over the points r of the elements whose support holds node i of N~_i(x_r) R_q[r], where R_q
// is the weighted sum of w(u^k) over the other dimensions' points (FP64 path: the chunk
// partials in rpart; tensor-core path: the tile partials in rpart_tc).
__device__ inline double gauss_row_integral(const StepParams& P, const Extra& X, int x, int i) {
  const Dim& dd = P.d[x];
  const int q = P.quad_q, s = (dd.b - 1) / 2;
  const int e0 = max(0, i - 1 - s), e1 = min(dd.n - 2, i + s);
  const int C = P.rchunks[x];
  double R = 0.0;
  for (int r = e0 * q; r < (e1 + 1) * q; ++r) {
    const int k = i - dd.phi0[r];
    if (k < 0 || k >= kPhiW) continue;
    const double ph = f2_to_double(dd.phi[static_cast<size_t>(r) * kPhiW + k]);
    if (ph == 0.0) continue;
    double rq = 0.0;
    if (P.precision == 0) {
      const double* rp = P.rpart + static_cast<size_t>(r) * C;
      for (int kk = 0; kk < C; ++kk) rq += rp[kk];
    } else {
      const TcDir& td = X.dirs[x];
      const long long T = static_cast<long long>(td.nrb) * td.ntc;
      const int rb = r / kTcM;
      const int Cr = tile_owner(T, P.vgrid, static_cast<long long>(rb) * td.ntc + td.ntc - 1) -
                     tile_owner(T, P.vgrid, static_cast<long long>(rb) * td.ntc) + 1;
      const double* rp = X.rpart_tc + static_cast<size_t>(r) * td.cmax;
      for (int kk = 0; kk < Cr; ++kk) rq += rp[kk];
    }
    R = fma(ph * dd.wq[r], rq, R);
  }
  return R;
}

// Right-hand side rows of this CTA's slice of direction x (Eq. KxQx), written as
// double-float into P.Q.  R_i (the nonlinear contraction, without L omega_i) comes from the
// partial buffers; the tensor-core partials lack the factor 4 a0 of w, and with cube (the cube
// form of the contraction) also the linear part -sum_j c_j u_ij = -sum_m a_m,i H_m (nodal
// rule; under the Gauss rule its Phi^T integral, sum_m (M a_m)_i H_m), which is added here
// from the same sums s1 starts with.
static __device__ __noinline__ void rhs_rows(const StepParams& P, const Extra& X, int x, int Mk, int M, int pb,
                         int cb, const Coef* c, bool cube = false) {
  const Dim& dd = P.d[x];
  int lo, hi;
  slice_of(dd.n, P.vgrid, P.vrank, lo, hi);
  const int rows = hi - lo;
  if (rows <= 0) return;
  // a group of tpr consecutive lanes per row; its lanes split the mode sums
  const int tpr = min(32, pow2_floor(max(1, kThreads / rows)));
  const int groups = kThreads / tpr, g = threadIdx.x / tpr, lane = threadIdx.x % tpr;
  const dfloat ct = ld_df(&P.ct_df), ck = ld_df(&P.ck_df), L = ld_df(&P.L_df);
  const int C = P.rchunks[x];
  const bool sep = sep_active(P, Mk);
  const int nsep = sep ? sep_terms(Mk) : 0;
  // contraction partials per row block (tensor-core path): a slice of rows shorter than a
  // block spans at most two row blocks; computed once (rb_lo < 0: per row)
  int rb_lo = 0, cr_lo = 0, cr_hi = 0;
  if (P.precision != 0 && !sep) {
    const TcDir& td = X.dirs[x];
    const long long T = static_cast<long long>(td.nrb) * td.ntc;
    rb_lo = lo / kTcM;
    const int rb_hi = (hi - 1) / kTcM;
    cr_lo = tile_owner(T, P.vgrid, static_cast<long long>(rb_lo) * td.ntc + td.ntc - 1) -
            tile_owner(T, P.vgrid, static_cast<long long>(rb_lo) * td.ntc) + 1;
    cr_hi = tile_owner(T, P.vgrid, static_cast<long long>(rb_hi) * td.ntc + td.ntc - 1) -
            tile_owner(T, P.vgrid, static_cast<long long>(rb_hi) * td.ntc) + 1;
    if (rb_hi > rb_lo + 1) rb_lo = -1;
  }
  for (int i0 = lo; i0 < hi; i0 += groups) {
    const int i = i0 + g;
    const bool live = i < hi;
    dfloat s1 = {0.f, 0.f}, s2 = {0.f, 0.f}, s3 = {0.f, 0.f}, s4 = {0.f, 0.f}, s5 = {0.f, 0.f};
    if (live) {
      // Gauss rule: M a and M b of the factors (consistent mass), nodal rule: a and b (the
      // diagonal mass joins below)
      const float2* Acol = P.quad ? dd.MA : dd.bank[pb];
      const float2* Bcol = P.quad ? dd.MB : dd.bank[cb];
      for (int m = lane; m < Mk; m += tpr) {
        const dfloat ami = ld_df(Acol + static_cast<size_t>(m) * dd.n + i), h = ld_df(c->H + m);
        s1 = df_fma(s1, ami, h);
        if (sep) s4 = df_add(s4, df_neg(df_mul(ami, h)));   // -u part of w (Eq. MxySep)
      }
      if (cube) s5 = s1;   // the cube form's linear part: sum_m a_m,i H_m
      // u^3 part of w: sum over multisets of a_m1 a_m2 a_m3 (row i of u^k's factors) T_q
      for (int q = lane; q < nsep; q += tpr) {
        const unsigned e = kSepTable.e[q];
        const dfloat a1 = ld_df(dd.bank[pb] + static_cast<size_t>(e & 0xFF) * dd.n + i);
        const dfloat a2 = ld_df(dd.bank[pb] + static_cast<size_t>((e >> 8) & 0xFF) * dd.n + i);
        const dfloat a3 = ld_df(dd.bank[pb] + static_cast<size_t>((e >> 16) & 0xFF) * dd.n + i);
        s4 = df_fma(s4, df_mul(df_mul(a1, a2), a3), ld_df(c->T + q));
      }
      for (int m = lane; m < M; m += tpr) {
        const dfloat bmi = ld_df(Bcol + static_cast<size_t>(m) * dd.n + i);
        const dfloat gm = ld_df(c->GM + m);
        s1 = df_add(s1, df_neg(df_mul(bmi, gm)));
        s2 = df_fma(s2, ld_df(dd.KB + static_cast<size_t>(m) * dd.n + i), gm);
        s3 = df_fma(s3, bmi, ld_df(c->GK + m));
      }
    }
    s1 = group_sum(s1, tpr);
    s2 = group_sum(s2, tpr);
    s3 = group_sum(s3, tpr);
    if (sep) s4 = group_sum(s4, tpr);
    if (cube) s5 = group_sum(s5, tpr);
    if (live && lane == 0) {
      dfloat R;
      if (sep) {
        R = df_mul(df_of(4.0 * P.a0), s4);
      } else if (P.quad) {
        R = df_of(gauss_row_integral(P, X, x, i));
        if (P.precision != 0) {
          if (cube) R = df_add(R, df_neg(s5));
          R = df_mul(df_of(4.0 * P.a0), R);
        }
      } else if (P.precision == 0) {
        const double* rp = P.rpart + static_cast<size_t>(i) * C;
        double r0 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
        int k = 0;
        for (; k + 3 < C; k += 4) { r0 += rp[k]; r1 += rp[k + 1]; r2 += rp[k + 2]; r3 += rp[k + 3]; }
        for (; k < C; ++k) r0 += rp[k];
        R = df_of((r0 + r1) + (r2 + r3));
      } else {
        const TcDir& td = X.dirs[x];
        const int rb = i / kTcM;
        int Cr;
        if (rb_lo < 0) {
          const long long T = static_cast<long long>(td.nrb) * td.ntc;
          Cr = tile_owner(T, P.vgrid, static_cast<long long>(rb) * td.ntc + td.ntc - 1) -
               tile_owner(T, P.vgrid, static_cast<long long>(rb) * td.ntc) + 1;
        } else {
          Cr = rb == rb_lo ? cr_lo : cr_hi;
        }
        // Slots of CTAs inside the row block's owner range that hold no tile of it are never
        // written: the buffer is zero between half-sweeps (cleared in the step prologue, and
        // every slot read here is cleared again for the next direction)
        double* rp = X.rpart_tc + static_cast<size_t>(i) * td.cmax;
        double part[8];   // loads first, so that their latencies overlap
#pragma unroll
        for (int k = 0; k < 8; ++k) part[k] = k < Cr ? rp[k] : 0.0;
        double r = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) r += part[k];
        for (int k = 8; k < Cr; ++k) r += rp[k];
        R = df_of(r);
        if (cube) R = df_add(R, df_neg(s5));
        R = df_mul(df_of(4.0 * P.a0), R);
        for (int k = 0; k < Cr; ++k) rp[k] = 0.0;
      }
      dfloat q;
      if (P.quad) {
        // Gauss rule: Q = c_t (M A H - M B GM) - c_k K B GM - c_k M B GK - L Phi^T (weighted sums)
        q = df_mul(ct, s1);
        q = df_add(q, df_neg(df_mul(ck, s2)));
        q = df_add(q, df_neg(df_mul(ck, s3)));
        q = df_add(q, df_neg(df_mul(L, R)));
      } else {
        const float2 om2 = kc_omega(X.kc[x], i);
        const dfloat om = {om2.x, om2.y};
        // Q = c_t om s1 - c_k s2 - c_k om s3 - L om R
        q = df_mul(df_mul(ct, om), s1);
        q = df_add(q, df_neg(df_mul(ck, s2)));
        q = df_add(q, df_neg(df_mul(df_mul(ck, om), s3)));
        q = df_add(q, df_neg(df_mul(df_mul(L, om), R)));
      }
      st_df(P.Q + i, q);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Grid of the nonlinear term: points per dimension and the FP64 weights of the fixed factors
// at those points (shared memory)
struct GridW {
  int n[kMaxDim];
  const double* w[kMaxDim];
};
__device__ __forceinline__ GridW nodal_grid(const StepParams& P, const double* wv) {
  GridW g;
  for (int d = 0; d < kMaxDim; ++d) {
    g.n[d] = d < P.dim ? P.d[d].n : 1;
    g.w[d] = wv + d * kMaxN;
  }
  return g;
}

// FP64 nonlinear contraction of the materialised w(u^k) grid (Eq. KxxMxx):
// rpart[c * C + k] = partial over chunk k of sum_{other indices} W * prod_{d != x} wv_d, with
// wv_d the weights of the fixed factors at the grid points: omega_d v_d (nodal rule), or
// omega_q,d (Phi_d v_d) at the Gauss points.
static __device__ __noinline__ void contract_fp64(const StepParams& P, int x, const GridW& g) {
  const int D = P.dim;
  const int n0 = g.n[0], n1 = g.n[1], n2 = D == 3 ? g.n[2] : 1;
  const int C = P.rchunks[x];
  const int nc = g.n[x];
  const int warp_g = P.vrank * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int total_warps = P.vgrid * kWarps;
  const double* W = P.W;
  if (D == 2 && (nc & 1) == 0 && (n0 & 1) == 0 && (n1 & 1) == 0) {
    // 2D with even extents: two adjacent grid values per 16-byte load, weights read from
    // shared memory (one broadcast read per row or column pair), two accumulator phases.
    // The FP64 pipe, not the issue slots, then bounds the pass.  The grid is read with the
    // streaming hint (evict first): it is larger than L2 and must not push out the small
    // working set of the other phases.
    const double2* W2 = reinterpret_cast<const double2*>(W);
    if (x == 1) {
      // column sums R[c] = sum_r W[r, c] wv0[r]; units (64-column block, row chunk)
      const int ncp = nc / 2;   // column pairs per row
      const int cblocks = (ncp + 31) / 32;
      const int units = cblocks * C;
      for (int u = warp_g; u < units; u += total_warps) {
        const int cb = u / C, k = u - cb * C;
        const int cp = cb * 32 + lane;
        int r0, r1;
        slice_of(n0, C, k, r0, r1);
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
        if (cp < ncp) {
          int r = r0;
          for (; r + 1 < r1; r += 2) {
            const double2 w0 = __ldcs(W2 + static_cast<size_t>(r) * ncp + cp);
            const double2 w1 = __ldcs(W2 + static_cast<size_t>(r + 1) * ncp + cp);
            const double f0 = g.w[0][r], f1 = g.w[0][r + 1];
            a0 = fma(w0.x, f0, a0);
            a1 = fma(w0.y, f0, a1);
            b0 = fma(w1.x, f1, b0);
            b1 = fma(w1.y, f1, b1);
          }
          if (r < r1) {
            const double2 w0 = __ldcs(W2 + static_cast<size_t>(r) * ncp + cp);
            a0 = fma(w0.x, g.w[0][r], a0);
            a1 = fma(w0.y, g.w[0][r], a1);
          }
          P.rpart[static_cast<size_t>(2 * cp) * C + k] = a0 + b0;
          P.rpart[static_cast<size_t>(2 * cp + 1) * C + k] = a1 + b1;
        }
      }
    } else {
      // row dots R[r] = sum_q W[r, q] wv1[q]; units (row, column chunk)
      const double2* wl2 = reinterpret_cast<const double2*>(g.w[1]);
      const int units = nc * C;
      for (int u = warp_g; u < units; u += total_warps) {
        const int c = u / C, k = u - c * C;
        int q0, q1;
        slice_of(n1 / 2, C, k, q0, q1);   // column pairs
        const double2* row = W2 + static_cast<size_t>(c) * (n1 / 2);
        double a0 = 0.0, a1 = 0.0;
        for (int q = q0 + lane; q < q1; q += 32) {
          const double2 w = __ldcs(row + q), f = wl2[q];
          a0 = fma(w.x, f.x, a0);
          a1 = fma(w.y, f.y, a1);
        }
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) P.rpart[static_cast<size_t>(c) * C + k] = acc;
      }
    }
    return;
  }
  if (x == D - 1) {
    // column sums: R[c] = sum_r W[r * nc + c] wrow(r); units (32-column block, row chunk)
    const int rows = static_cast<int>(static_cast<long long>(n0) * n1 * n2 / nc);
    const int cblocks = (nc + 31) / 32;
    const int units = cblocks * C;
    for (int u = warp_g; u < units; u += total_warps) {
      const int cb = u / C, k = u - cb * C;
      const int c = cb * 32 + lane;
      int r0, r1;
      slice_of(rows, C, k, r0, r1);
      double acc = 0.0;
      for (int rb = r0; rb < r1; rb += 32) {
        const int r = rb + lane;
        double wr = 0.0;
        if (r < r1) wr = (D == 2) ? g.w[0][r] : g.w[0][r / n1] * g.w[1][r % n1];
        const int cnt = min(32, r1 - rb);
        for (int t = 0; t < cnt; ++t) {
          const double w = __shfl_sync(0xffffffffu, wr, t);
          if (c < nc) acc = fma(W[static_cast<size_t>(rb + t) * nc + c], w, acc);
        }
      }
      if (c < nc) P.rpart[static_cast<size_t>(c) * C + k] = acc;
    }
  } else {
    // row dots over the last axis
    const int nl = (D == 2) ? n1 : n2;
    const double* wl = g.w[D - 1];   // weights of the last dimension
    const int units = nc * C;
    for (int u = warp_g; u < units; u += total_warps) {
      const int c = u / C, k = u - c * C;
      double acc = 0.0;
      if (D == 2) {          // x = 0: one row per c, chunk over the last axis
        int q0, q1;
        slice_of(nl, C, k, q0, q1);
        const double* row = W + static_cast<size_t>(c) * nl;
        for (int q = q0 + lane; q < q1; q += 32) acc = fma(row[q], wl[q], acc);
      } else {               // D == 3, x in {0, 1}: rows over the other leading dimension
        const int no = (x == 0) ? n1 : n0;
        const double* wo = g.w[(x == 0) ? 1 : 0];
        int i0, i1;
        slice_of(no, C, k, i0, i1);
        for (int i = i0; i < i1; ++i) {
          const size_t base = (x == 0) ? (static_cast<size_t>(c) * n1 + i) * nl
                                       : (static_cast<size_t>(i) * n1 + c) * nl;
          double s = 0.0;
          for (int q = lane; q < nl; q += 32) s = fma(W[base + q], wl[q], s);
          acc = fma(wo[i], s, acc);
        }
      }
      acc = warp_sum(acc);
      if (lane == 0) P.rpart[static_cast<size_t>(c) * C + k] = acc;
    }
  }
}

// FP64 weights omega_d v_d of every dimension but x (shared memory wv + d * kMaxN).
static __device__ __noinline__ void load_weights_fp64(const StepParams& P, const Extra& X, int x, double* wv) {
  for (int d = 0; d < P.dim; ++d) {
    if (d == x) continue;
    const Dim& dd = P.d[d];
    constexpr int kGroup = 8;   // loads first, so that their latencies overlap
    for (int i0 = threadIdx.x; i0 < dd.n; i0 += kGroup * blockDim.x) {
      double om[kGroup];
      float2 v[kGroup];
#pragma unroll
      for (int g = 0; g < kGroup; ++g) {
        const int i = i0 + g * blockDim.x;
        om[g] = i < dd.n ? dd.omega[i] : 0.0;
        v[g] = i < dd.n ? dd.v[i] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int g = 0; g < kGroup; ++g) {
        const int i = i0 + g * blockDim.x;
        if (i < dd.n) wv[d * kMaxN + i] = om[g] * f2_to_double(v[g]);
      }
    }
  }
  __syncthreads();
}

// Gauss rule: FP64 weights omega_q,d (Phi_d v_d) of every dimension but x at its Gauss points,
// packed in shared memory (each dimension's block at an even offset, for 16-byte loads).  The
// host admits the rule only when the blocks fit the phase's kMaxDim * kMaxN doubles.
static __device__ __noinline__ GridW load_weights_gauss(const StepParams& P, int x, double* wv) {
  GridW g;
  int off = 0;
  for (int d = 0; d < kMaxDim; ++d) {
    g.n[d] = d < P.dim ? P.d[d].nq : 1;
    g.w[d] = wv;
    if (d >= P.dim || d == x) continue;
    const Dim& dd = P.d[d];
    g.w[d] = wv + off;
    const int phiw = dd.b + 1;
    for (int r = threadIdx.x; r < dd.nq; r += blockDim.x)
      wv[off + r] = dd.wq[r] * df_to_double(phi_row(dd, phiw, dd.v, r));
    off += (dd.nq + 1) & ~1;
  }
  __syncthreads();
  return g;
}

// Gauss rule, step prologue (own slices): u^k's factors at the Gauss points, Aq = Phi a, and
// the consistent-mass products M a (double-float), for the right-hand sides and the grid.
static __device__ __noinline__ void gauss_prologue(const StepParams& P, const Extra& X, int pb, int Mk) {
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    const int phiw = dd.b + 1;
    int lo, hi;
    slice_of(dd.nq, P.vgrid, P.vrank, lo, hi);
    for (int m = 0; m < Mk; ++m) {
      const float2* col = dd.bank[pb] + static_cast<size_t>(m) * dd.n;
      for (int r = lo + threadIdx.x; r < hi; r += blockDim.x)
        st_df(dd.Aq + static_cast<size_t>(m) * dd.nq + r, phi_row(dd, phiw, col, r));
    }
    slice_of(dd.n, P.vgrid, P.vrank, lo, hi);
    for (int m = 0; m < Mk; ++m) {
      const float2* col = dd.bank[pb] + static_cast<size_t>(m) * dd.n;
      for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        st_df(dd.MA + static_cast<size_t>(m) * dd.n + i, mv_row(X.kc[d], col, i));
    }
  }
}

// Gauss rule: W = w(u^k) on the grid of Gauss points from the factors at the points Aq (FP64
// reconstruction; row-major grid).
static __device__ __noinline__ void materialise_w_gauss(const StepParams& P, int Mk) {
  const int D = P.dim;
  const int n0 = P.d[0].nq, n1 = P.d[1].nq, n2 = D == 3 ? P.d[2].nq : 1;
  const long long N = static_cast<long long>(n0) * n1 * n2;
  const long long stride = static_cast<long long>(P.vgrid) * blockDim.x;
  for (long long p = static_cast<long long>(P.vrank) * blockDim.x + threadIdx.x; p < N; p += stride) {
    const int l = static_cast<int>(p % n2);
    const long long ij = p / n2;
    const int j = static_cast<int>(ij % n1), i = static_cast<int>(ij / n1);
    double u = 0.0;
    for (int m = 0; m < Mk; ++m) {
      double t = f2_to_double(P.d[0].Aq[static_cast<size_t>(m) * n0 + i]) *
                 f2_to_double(P.d[1].Aq[static_cast<size_t>(m) * n1 + j]);
      if (D == 3) t *= f2_to_double(P.d[2].Aq[static_cast<size_t>(m) * n2 + l]);
      u += t;
    }
    __stcs(P.W + p, 4.0 * P.a0 * (u * u * u - u));
  }
}

// Adaptive CTD, step from the full-grid field U (nodal rule): the whole right-hand side from
// u^k, c_t M u^k - int N~ L w(u^k), is one full-grid term; W = w(U) - (c_t / L) U makes the
// contraction's -L omega R carry both parts (the step has no factors of u^k).
static __device__ __noinline__ void materialise_w_grid(const StepParams& P) {
  const int D = P.dim;
  const long long N = static_cast<long long>(P.d[0].n) * P.d[1].n * (D == 3 ? P.d[2].n : 1);
  const long long stride = static_cast<long long>(P.vgrid) * blockDim.x;
  const double r = P.c_t / P.L;
  for (long long p = static_cast<long long>(P.vrank) * blockDim.x + threadIdx.x; p < N; p += stride) {
    const double u = P.U[p];
    __stcs(P.W + p, 4.0 * P.a0 * (u * u * u - u) - r * u);
  }
}

// Reduced integration domain: the grid is cut into blocks of 128 nodes per dimension (the
// tensor-core tile edge; a 3D tile of direction x lies inside one block), numbered row-major
// over the blocks of dimensions 0, 1 (, 2).
struct RdBlocks {
  int n[3], nb[3];
  __device__ explicit RdBlocks(const StepParams& P) {
    for (int d = 0; d < 3; ++d) {
      n[d] = d < P.dim ? P.d[d].n : 1;
      nb[d] = d < P.dim ? (n[d] + kTcM - 1) / kTcM : 1;
    }
  }
  __device__ int count() const { return nb[0] * nb[1] * nb[2]; }
  // block blk: node ranges [lo[d], hi[d])
  __device__ void range(int blk, int (&lo)[3], int (&hi)[3]) const {
    int b[3];
    b[2] = blk % nb[2];
    b[1] = (blk / nb[2]) % nb[1];
    b[0] = blk / (nb[2] * nb[1]);
    for (int d = 0; d < 3; ++d) {
      lo[d] = b[d] * kTcM;
      hi[d] = min(n[d], lo[d] + kTcM);
      if (nb[d] == 1 && n[d] == 1) { lo[d] = 0; hi[d] = 1; }
    }
  }
};

// FP64 path: every block whose largest |W| is not above reduced_tol is set to zero.  Blocks are
// split over the CTAs; each CTA reads its block, reduces the maximum in a fixed order, then
// zeroes it.
static __device__ __noinline__ void reduce_domain_fp64(const StepParams& P) {
  const RdBlocks B(P);
  double* W = P.W;
  __shared__ double s_red[kWarps];
  __shared__ int s_keep;
  for (int blk = P.vrank; blk < B.count(); blk += P.vgrid) {
    int lo[3], hi[3];
    B.range(blk, lo, hi);
    const int w1 = hi[1] - lo[1], w2 = hi[2] - lo[2], cnt = (hi[0] - lo[0]) * w1 * w2;
    auto at = [&](int e) -> size_t {
      const int l = lo[2] + e % w2, j = lo[1] + (e / w2) % w1, i = lo[0] + e / (w2 * w1);
      return (static_cast<size_t>(i) * B.n[1] + j) * B.n[2] + l;
    };
    double mx = 0.0;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) mx = fmax(mx, fabs(W[at(e)]));
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int k = 0; k < kWarps; ++k) m = fmax(m, s_red[k]);
      s_keep = m > P.reduced_tol;
    }
    __syncthreads();
    if (!s_keep)
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) W[at(e)] = 0.0;
    __syncthreads();
  }
}

// Tensor-core path: max |u(u^2 - 1)| of u^k over every block, from the FP32 parts of the
// factors (the arithmetic of the tiles it gates), into P.tile_max (float bits).  Blocks are
// split over the CTAs; a block's factor rows are staged in shared memory (sh: D * 128 * Mk
// floats).
static __device__ __noinline__ void classify_tiles(const StepParams& P, int pb, int Mk, float* sh) {
  const RdBlocks B(P);
  const int D = P.dim;
  float* sf[3] = {sh, sh + Mk * kTcM, sh + 2 * Mk * kTcM};   // [Mk][128] per dimension
  __shared__ float s_red[kWarps];
  for (int blk = P.vrank; blk < B.count(); blk += P.vgrid) {
    int lo[3], hi[3];
    B.range(blk, lo, hi);
    __syncthreads();
    for (int d = 0; d < D; ++d) {
      const Dim& dd = P.d[d];
      for (int e = threadIdx.x; e < Mk * kTcM; e += blockDim.x) {
        const int m = e / kTcM, r = e - m * kTcM, i = lo[d] + r;
        const float2 a = i < hi[d] ? dd.bank[pb][static_cast<size_t>(m) * dd.n + i] : make_float2(0.f, 0.f);
        sf[d][e] = a.x + a.y;
      }
    }
    __syncthreads();
    const int w1 = hi[1] - lo[1], w2 = hi[2] - lo[2], cnt = (hi[0] - lo[0]) * w1 * w2;
    float mx = 0.f;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int l = e % w2, j = (e / w2) % w1, i = e / (w2 * w1);
      float u = 0.f;
      if (D == 2) {
        for (int m = 0; m < Mk; ++m) u = __fmaf_rn(sf[0][m * kTcM + i], sf[1][m * kTcM + j], u);
      } else {
        for (int m = 0; m < Mk; ++m) u = __fmaf_rn(sf[0][m * kTcM + i] * sf[1][m * kTcM + j], sf[2][m * kTcM + l], u);
      }
      mx = fmaxf(mx, fabsf(u * __fmaf_rn(u, u, -1.f)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float m = 0.f;
      for (int k = 0; k < kWarps; ++k) m = fmaxf(m, s_red[k]);
      P.tile_max[blk] = __float_as_uint(m);
    }
  }
  __syncthreads();
}

// w(u) = dF/du = 4 a0 (u^3 - u) (Eq. energyfunction)
__device__ __forceinline__ double w_of_u(double u, double a0) { return 4.0 * a0 * (u * u * u - u); }

// Materialise W = w(u^k) on the grid from FP64 factor copies Af[d][m][i] (row-major grid).
static __device__ __noinline__ void materialise_w(const StepParams& P, const Extra& X, int Mk) {
  const int D = P.dim;
  const int n0 = P.d[0].n, n1 = P.d[1].n, n2 = D == 3 ? P.d[2].n : 1;
  const long long N = static_cast<long long>(n0) * n1 * n2;
  const long long stride = static_cast<long long>(P.vgrid) * blockDim.x;
  for (long long p = static_cast<long long>(P.vrank) * blockDim.x + threadIdx.x; p < N; p += stride) {
    double u = 0.0;
    if (D == 2) {
      // 32-bit index arithmetic (N < 2^31 for every 2D grid of up to kMaxN^2 nodes)
      const unsigned pu = static_cast<unsigned>(p);
      const int i = static_cast<int>(pu / static_cast<unsigned>(n1)), j = static_cast<int>(pu - static_cast<unsigned>(i) * n1);
      for (int m = 0; m < Mk; ++m)
        u = fma(X.Af[0][static_cast<size_t>(m) * n0 + i], X.Af[1][static_cast<size_t>(m) * n1 + j], u);
    } else {
      const int l = static_cast<int>(p % n2);
      const long long ij = p / n2;
      const int j = static_cast<int>(ij % n1), i = static_cast<int>(ij / n1);
      for (int m = 0; m < Mk; ++m)
        u = fma(X.Af[0][static_cast<size_t>(m) * n0 + i] * X.Af[1][static_cast<size_t>(m) * n1 + j],
                X.Af[2][static_cast<size_t>(m) * n2 + l], u);
    }
    __stcs(P.W + p, w_of_u(u, P.a0));   // streaming store: the grid exceeds L2
  }
}

}  // namespace ctd

// Kernels of the CTD step: the persistent per-step kernel (Section 3.3 solution algorithm,
// all control on the device), the discrete energy, and probe kernels for single stages.
#include <algorithm>
#include <cstdio>

#include "ctd_kernels.h"
#include "ctd_step.cuh"

// Functions the separated-form translation unit compiles again get internal linkage there
#ifdef CTD_SEPARATED_TU
#define CTD_LOCAL static
#else
#define CTD_LOCAL
#endif

namespace ctd {

// ---------------------------------------------------------------------------------------
// Shared-memory plan of the step kernel (one union over phases)
// Fixed part; the per-phase arena follows it:
//   Phase A: Gram row data (3 * kChunk float2) or FP64 weights (kMaxDim * kMaxN doubles)
//   Phase C: solution (n_max float2) then, if they fit, the solver factors.
struct SmemStep {
  Coef coef;
  float2 red2[2 * kMaxDim];
  float redf[kWarps];
};
constexpr size_t kArenaOffset = (sizeof(SmemStep) + 127) / 128 * 128;
__host__ __device__ inline size_t arena_phase_a_bytes() {
  return sizeof(double) * kMaxDim * kMaxN > sizeof(float2) * 3 * kChunk ? sizeof(double) * kMaxDim * kMaxN
                                                                         : sizeof(float2) * 3 * kChunk;
}
static_assert(kCoefScratchBytes <= sizeof(double) * kMaxDim * kMaxN, "coefficient scratch exceeds the arena");
__host__ __device__ inline size_t solver_smem_offset(int n_max) { return (sizeof(float2) * n_max + 127) / 128 * 128; }

struct Arena {
  float2* gram_rows;
  double* wv;
  float2* xsol;
  float* solver;
};
__device__ inline unsigned char* arena_base(unsigned char* smem_raw) {
  const uint32_t s0 = smem_u32(smem_raw);
  const uint32_t a = (s0 + static_cast<uint32_t>(kArenaOffset) + 1023u) & ~1023u;
  return smem_raw + (a - s0);
}
__device__ inline Arena arena_of(unsigned char* smem_raw, const StepParams& P) {
  unsigned char* a = arena_base(smem_raw);
  Arena r;
  r.gram_rows = reinterpret_cast<float2*>(a);
  r.wv = reinterpret_cast<double*>(a);
  r.xsol = reinterpret_cast<float2*>(a);
  // Phase C: mode 0 -> [x (n_max float2)][factors]; mode 1 -> [level-1 factors], x global;
  // mode 2 -> [x], factors global
  if (P.solver_mode == 0 || P.solver_mode == 3) {
    r.solver = reinterpret_cast<float*>(a + solver_smem_offset(P.n_max));
  } else if (P.solver_mode == 1) {
    r.solver = reinterpret_cast<float*>(a);
    r.xsol = P.xsol_g;
  } else {
    r.solver = P.solver;
  }
  return r;
}

// Kernel parameter blocks are indexed with runtime dimension numbers; staged in shared memory
// they stay addressable without a per-thread local copy.
template <typename T>
__device__ __forceinline__ void stage_to_smem(T* dst, const T& src) {
  const int* s = reinterpret_cast<const int*>(&src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(T) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

// Shared-memory copy of the parameters with this CTA's place in the virtual grid
__device__ __forceinline__ void stage_params(StepParams* dst, const StepParams& src, int vgrid, int vrank) {
  stage_to_smem(dst, src);
  __syncthreads();
  if (threadIdx.x == 0) {
    dst->vgrid = vgrid;
    dst->vrank = vrank;
  }
}

__device__ __forceinline__ void trace_mark(const StepParams& P, unsigned long long& t, int phase) {
  if (P.trace && P.vrank == 0 && threadIdx.x == 0) {
    const unsigned long long now = global_ns();
    atomicAdd(P.trace + phase, now - t);
    t = now;
  }
}

__device__ inline bool sync_all(const StepParams& P, unsigned& epoch, int where) {
  if (P.vgrid == 1) {
    __syncthreads();
    return true;
  }
  return grid_barrier(P.barrier, epoch, P.wait_ns, P.st, where);
}

// Convert u^k factors of this CTA's slices to FP64 copies (FP64-path materialisation).
CTD_LOCAL __device__ __noinline__ void convert_prev_modes(const StepParams& P, const Extra& X, int pb, int Mk) {
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    int lo, hi;
    slice_of(dd.n, P.vgrid, P.vrank, lo, hi);
    for (int m = 0; m < Mk; ++m)
      for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        X.Af[d][static_cast<size_t>(m) * dd.n + i] = f2_to_double(dd.bank[pb][static_cast<size_t>(m) * dd.n + i]);
  }
}

// Mode start vectors (own slices): warm start from u^k's mode m if present and not zero,
// otherwise SplitMix64 entries in [0.5, 1.5).
CTD_LOCAL __device__ __noinline__ void init_mode(const StepParams& P, int m, int pb, int Mk, long long step) {
  __shared__ int s_nz[kMaxDim];
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    int nz = 0;
    if (m < Mk) {
      const float2* col = dd.bank[pb] + static_cast<size_t>(m) * dd.n;
      for (int i = threadIdx.x; i < dd.n; i += blockDim.x)
        if (col[i].x != 0.f || col[i].y != 0.f) nz = 1;
    }
    nz = __syncthreads_or(nz);
    if (threadIdx.x == 0) s_nz[d] = nz;
  }
  __syncthreads();
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    int lo, hi;
    slice_of(dd.n, P.vgrid, P.vrank, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      float2 v;
      if (s_nz[d]) {
        v = dd.bank[pb][static_cast<size_t>(m) * dd.n + i];
      } else {
        const dfloat r = df_from_double(mode_init_value(P.seed, step, m, d, i));
        v = make_float2(r.hi, r.lo);
      }
      dd.v[i] = v;
    }
  }
}

// Convergence partials (own slices): per dimension c the six products of old, delta = new -
// old and new, and max |new|; slot (c * 6 + k) of the gram buffer, maxpart[c * G + cta].
CTD_LOCAL __device__ __noinline__ void convergence_partials(const StepParams& P, const Extra& X, float2* sh) {
  const int G = gram_ctas(P), cta = P.vrank;
  if (cta >= G) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < P.dim; ++c) {
    const Dim& dd = P.d[c];
    int lo, hi;
    slice_of(dd.n, G, cta, lo, hi);
    dfloat a[6];
    for (int k = 0; k < 6; ++k) a[k] = {0.f, 0.f};
    double mx = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const dfloat nv = ld_df(dd.v + i);
      const dfloat od = ld_df(dd.vold + i);
      const dfloat dl = df_add(nv, df_neg(od));
      a[0] = df_fma(a[0], od, od);
      a[1] = df_fma(a[1], od, dl);
      a[2] = df_fma(a[2], od, nv);
      a[3] = df_fma(a[3], dl, dl);
      a[4] = df_fma(a[4], dl, nv);
      a[5] = df_fma(a[5], nv, nv);
      mx = fmax(mx, fabs(df_to_double(nv)));
    }
    for (int k = 0; k < 6; ++k) {
      const dfloat r = group_sum(a[k], 32);
      if (lane == 0) st_df(sh + warp * 6 + k, r);
    }
    mx = warp_max(mx);
    __shared__ double s_mx[kWarps];
    if (lane == 0) s_mx[warp] = mx;
    __syncthreads();
    if (threadIdx.x < 6) {
      dfloat s = {0.f, 0.f};
      for (int w = 0; w < kWarps; ++w) s = df_add(s, ld_df(sh + w * 6 + threadIdx.x));
      st_df(P.gram + static_cast<size_t>(c * 6 + threadIdx.x) * G + cta, s);
    }
    if (threadIdx.x == 6) {
      double m = 0.0;
      for (int w = 0; w < kWarps; ++w) m = fmax(m, s_mx[w]);
      X.maxpart[c * G + cta] = m;
    }
    __syncthreads();
  }
}

// Gauss rule, tensor-core path: the point rows' tile partials are read by several nodes'
// right-hand sides, so they are cleared after the right-hand sides (during the solve, by the
// CTAs that do not solve), not as they are read.
CTD_LOCAL __device__ __noinline__ void clear_point_partials(const StepParams& P, const Extra& X, int x) {
  const int parts = P.vgrid > 1 ? P.vgrid - 1 : 1, me = P.vgrid > 1 ? P.vrank - 1 : 0;
  if (me < 0) return;
  const size_t total = static_cast<size_t>(P.d[x].nq) * X.dirs[x].cmax;
  int lo, hi;
  slice_of(static_cast<int>(total), parts, me, lo, hi);
  for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) X.rpart_tc[i] = 0.0;
}

// Save the current trial factors (own slices) at the start of a sweep.
CTD_LOCAL __device__ __noinline__ void save_old(const StepParams& P) {
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    int lo, hi;
    slice_of(dd.n, P.vgrid, P.vrank, lo, hi);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) dd.vold[i] = dd.v[i];
  }
}

// Commit the converged mode (own slices): b = v * scale_d, K b.
CTD_LOCAL __device__ __noinline__ void commit_mode(const StepParams& P, const Extra& X, int M, int cb,
                            const double* scale) {
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    int lo, hi;
    slice_of(dd.n, P.vgrid, P.vrank, lo, hi);
    const dfloat sc = df_of(scale[d]);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      st_df(dd.bank[cb] + static_cast<size_t>(M) * dd.n + i, df_mul(ld_df(dd.v + i), sc));
      st_df(dd.KB + static_cast<size_t>(M) * dd.n + i, df_mul(kv_row(X.kc[d], dd.v, i), sc));
      if (P.quad) st_df(dd.MB + static_cast<size_t>(M) * dd.n + i, df_mul(mv_row(X.kc[d], dd.v, i), sc));
    }
  }
}

// The solver CTA: solve Eq. ux for direction x, normalise unless x is the last dimension,
// publish v_x (double-float) and flags in ctrl: [0] zero factor, [1] failure.
CTD_LOCAL __device__ __noinline__ void solve_direction(const StepParams& P, const Extra& X, int x, SmemStep& sm,
                                const Arena& ar, bool warm, float tau0) {
  const Dim& dd = P.d[x];
  const SolverStore store = solver_bind(P.solver_mode == 2 ? 0 : P.solver_mode, ar.solver, P.solver, dd.n, dd.b, dd.mu_max);
  const dfloat a1 = ld_df(&sm.coef.alpha1), a2 = ld_df(&sm.coef.alpha2);
  float2* xs = ar.xsol;
  float2* prev = X.xprev + static_cast<size_t>(x) * kMaxN;
  bool ok = banded_solve(store, X.kc[x], a1, a2, P.Q, xs, sm.redf, P.trace, warm ? prev : nullptr,
                         P.precision != 0 ? kSolveTolMixed : kSolveTolFp64, tau0);
  for (int i = threadIdx.x; i < dd.n; i += blockDim.x) prev[i] = xs[i];
  // zero test and squared norm (double-float, fixed reduction order)
  int nz = 0;
  dfloat ss = {0.f, 0.f};
  for (int i = threadIdx.x; i < dd.n; i += blockDim.x) {
    const dfloat v = {xs[i].x, xs[i].y};
    if (v.hi != 0.f || v.lo != 0.f) nz = 1;
    ss = df_fma(ss, v, v);
  }
  nz = __syncthreads_or(nz);
  ss = group_sum(ss, 32);
  __shared__ float2 s_part[kWarps];
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = make_float2(ss.hi, ss.lo);
  __syncthreads();
  __shared__ double s_inv;
  if (threadIdx.x == 0) {
    dfloat t = {0.f, 0.f};
    for (int w = 0; w < kWarps; ++w) t = df_add(t, ld_df(s_part + w));
    const double nrm = sqrt(df_to_double(t));
    s_inv = (nz && x != P.dim - 1) ? 1.0 / nrm : 1.0;
    if (!(nrm == nrm) || nrm > 1e300) ok = false;
    X.ctrl[0] = nz ? 0 : 1;
    X.ctrl[1] = ok ? 0 : 1;
  }
  __syncthreads();
  const dfloat inv = df_of(s_inv);
  for (int i = threadIdx.x; i < dd.n; i += blockDim.x) {
    dfloat v = {xs[i].x, xs[i].y};
    if (x != P.dim - 1) v = df_mul(v, inv);
    st_df(dd.v + i, v);
  }
}

// ---------------------------------------------------------------------------------------
CTD_LOCAL __device__ void step_body(const StepParams& P, const Extra& X, unsigned char* smem_raw,
                          uint32_t tmem_base) {
  SmemStep& sm = *reinterpret_cast<SmemStep*>(smem_raw);
  const Arena ar = arena_of(smem_raw, P);
  unsigned epoch = 0;
  unsigned long long tmark = global_ns();
  const InstState st0 = *P.st;
  if (st0.status != 0) return;
  const int D = P.dim, pb = st0.bank, cb = 1 - pb, Mk = st0.Mk;

  // ---- prologue: the nonlinear term's data for this step (none for the separated form,
  // whose 1D sums are Gram slots)
  bool cube = false;
  if constexpr (kSepTU) {
  } else if (P.precision == 0) {
    convert_prev_modes(P, X, pb, Mk);
    if (P.quad) gauss_prologue(P, X, pb, Mk);
    if (!sync_all(P, epoch, 1)) return;
    if (st0.grid) materialise_w_grid(P);   // adaptive CTD: u^k held on the full grid
    else if (P.quad) materialise_w_gauss(P, Mk);
    else materialise_w(P, X, Mk);
  } else {
    if (P.quad) {
      gauss_prologue(P, X, pb, Mk);
      if (!sync_all(P, epoch, 1)) return;
    }
    // the cube form of the contraction (see tc_amp_bound): the reduced domain drops tiles of
    // w(u), which the cube form does not hold apart from the linear part, so it keeps the
    // direct form
    if (Mk > 0 && P.reduced_tol <= 0.0 && P.contraction_form != 1)
      cube = P.contraction_form == 2 ||
             tc_amp_bound(P, pb, Mk, reinterpret_cast<float*>(arena_base(smem_raw))) <= kCubeMaxAmp;
    tc_prepare(P, X.dirs, X.kr, pb, Mk, !cube);
    fence_proxy_async_global();
    // contraction partial slots start the step at zero (see rhs_rows)
    size_t nslot = 0;
    for (int d = 0; d < D; ++d) {
      const size_t v = static_cast<size_t>(P.d[d].nq) * X.dirs[d].cmax;
      nslot = v > nslot ? v : nslot;
    }
    for (size_t i = static_cast<size_t>(P.vrank) * blockDim.x + threadIdx.x; i < nslot;
         i += static_cast<size_t>(P.vgrid) * blockDim.x)
      X.rpart_tc[i] = 0.0;
  }
  if (!kSepTU && P.reduced_tol > 0.0 && Mk > 0) {
    // reduced integration domain (Section 3.3): the nonlinear term is fixed for the step, so
    // its 128 x 128 node blocks are classified once
    if (P.precision == 0) {
      if (!sync_all(P, epoch, 9)) return;
      reduce_domain_fp64(P);
    } else {
      classify_tiles(P, pb, Mk, reinterpret_cast<float*>(arena_base(smem_raw)));
    }
  }
  trace_mark(P, tmark, kTrPrologue);

  int M = 0, sweeps = 0, sweeps_max = 0, not_conv = 0, n_stalled = 0, sweeps_discarded = 0;
  double amp0 = 0.0;   // amplitude max|(x)v| of the step's leading mode
  bool stopped = false;
  // adaptive CTD: a budget of M_c + 1 modes; committing the last one means M > M_c
  const int n_modes = P.fixed_modes > 0 ? P.fixed_modes
                                        : (P.actd_Mc > 0 && P.actd_Mc < P.M_max ? P.actd_Mc + 1 : P.M_max);
  const int n_it = P.fixed_als > 0 ? P.fixed_als : P.I_max;
  for (int m = 0; m < n_modes; ++m) {
    init_mode(P, m, pb, Mk, st0.step);
    if (!sync_all(P, epoch, 2)) return;
    trace_mark(P, tmark, kTrInit);
    bool zero_mode = false;
    double delta = 1e300, amp = 0.0, delta_prev = 1e300;
    double norms2[kMaxDim] = {1.0, 1.0, 1.0};
    int it;
    for (it = 1; it <= n_it; ++it) {
      save_old(P);
      for (int x = 0; x < D; ++x) {
        if (cube) {
          // cube form: the column operand scaled by the cube roots of the current weights
          tc_prepare_scaled(P, X.kc, X.dirs[x], X.kr[x], pb, Mk, reinterpret_cast<float*>(arena_base(smem_raw)));
          fence_proxy_async_global();
          if (!sync_all(P, epoch, 14)) return;
          trace_mark(P, tmark, kTrScale);
        }
        // Phase A: Gram partials of the fixed factors + nonlinear contraction partials
        unsigned long long tsub = (P.trace && P.vrank == 0 && threadIdx.x == 0) ? global_ns() : 0ull;
        gram_partials(P, X, x, Mk, M, pb, cb, ar.gram_rows);
        __syncthreads();
        if (P.trace && P.vrank == 0 && threadIdx.x == 0) {
          const unsigned long long t = global_ns();
          atomicAdd(P.trace + kTrGram, t - tsub);
        }
        // the contraction is timed on the last CTA, which has a full tile share
        const bool tr_last = P.trace && P.vrank == P.vgrid - 1 && threadIdx.x == 0;
        const unsigned long long tcon = tr_last ? global_ns() : 0ull;
        if constexpr (kSepTU) {
        } else if (P.precision == 0) {
          GridW g;
          if (P.quad) {
            g = load_weights_gauss(P, x, ar.wv);
          } else {
            load_weights_fp64(P, X, x, ar.wv);
            g = nodal_grid(P, ar.wv);
          }
          contract_fp64(P, x, g);
        } else {
          const TcDir& td = X.dirs[x];
          const __nv_bfloat16* qop = (D == 2 && !cube) ? P.d[td.last].op : X.kr[x];
          if (!tc_contract(P, X.kc, td, P.d[x].op, qop, x, Mk, X.tc_stages, arena_base(smem_raw), tmem_base,
                           X.rpart_tc, nullptr, P.reduced_tol > 0.0 ? P.tile_max : nullptr,
                           static_cast<float>(4.0 * P.a0), static_cast<float>(P.reduced_tol), cube))
            return;
        }
        if (tr_last) atomicAdd(P.trace + kTrContract, global_ns() - tcon);
        if (!sync_all(P, epoch, 3)) return;
        trace_mark(P, tmark, kTrGramContract);
        // Phase B: coefficients (every CTA, same order) and right-hand-side rows
        build_coefficients(P, x, Mk, M, &sm.coef, ar.gram_rows);
        rhs_rows(P, X, x, Mk, M, pb, cb, &sm.coef, cube);
        if (!sync_all(P, epoch, 4)) return;
        trace_mark(P, tmark, kTrRhs);
        // Phase C: banded solve on CTA 0
        // tensor-core path: a warm start from the previous sweep is off by about the mode's last
        // relative change, so the first pass only needs tol / (4 delta) of error reduction
        float tau0 = kFirstPassTau;
        if (P.precision != 0 && it > 1 && delta < 1e299)
          tau0 = fminf(fmaxf(static_cast<float>(kSolveTolMixed / (4.0 * fmax(delta, 1e-30))), kFirstPassTau),
                       3.90625e-3f);
        if (P.vrank == 0) solve_direction(P, X, x, sm, ar, it > 1, tau0);
        if (!kSepTU && P.quad && P.precision != 0) clear_point_partials(P, X, x);
        if (!sync_all(P, epoch, 5)) return;
        trace_mark(P, tmark, kTrSolve);
        const int zflag = *reinterpret_cast<volatile int*>(X.ctrl + 0);
        const int fflag = *reinterpret_cast<volatile int*>(X.ctrl + 1);
        if (fflag) {
          if (P.vrank == 0 && threadIdx.x == 0) atomicOr(&P.st->status, kErrNonfinite);
          return;
        }
        if (zflag) { zero_mode = true; break; }
      }
      ++sweeps;
      if (zero_mode) break;
      // Phase D: relative change of the rank-1 mode, max entries, norms
      convergence_partials(P, X, ar.gram_rows);
      if (!sync_all(P, epoch, 6)) return;
      trace_mark(P, tmark, kTrConverge);
      {
        __shared__ double s_dots[kMaxDim * 6];
        __shared__ double s_max[kMaxDim];
        // the D * 6 dot slots and D max slots: 16 lanes per slot, lane g holds CTA g's
        // partial; all loads issued together, then fixed xor trees
        const int Gg = gram_ctas(P);
        const int g = threadIdx.x & 15, sub = threadIdx.x >> 4, nd = D * 6, nu = nd + D;
        float2 pv[2];
        double pm[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int u = r * (kThreads / 16) + sub;
          pv[r] = make_float2(0.f, 0.f);
          pm[r] = 0.0;
          if (g < Gg && u < nd) pv[r] = P.gram[static_cast<size_t>(u) * Gg + g];
          else if (g < Gg && u < nu) pm[r] = X.maxpart[(u - nd) * Gg + g];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int u = r * (kThreads / 16) + sub;
          const dfloat t = group_sum(dfloat{pv[r].x, pv[r].y}, 16);
          double mx = pm[r];
          for (int o = 8; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          if (g == 0 && u < nd) s_dots[u] = df_to_double(t);
          else if (g == 0 && u < nu) s_max[u - nd] = mx;
        }
        __syncthreads();
        // ||(x)new - (x)old||^2 = sum_{d,e} prod_c <T_d(c), T_e(c)>, factor of T_d at c:
        // old (c < d), delta (c == d), new (c > d); dot index table over {old, delta, new}
        const int idx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        double num = 0.0, den = 1.0;
        for (int d1 = 0; d1 < D; ++d1)
          for (int e1 = 0; e1 < D; ++e1) {
            double prod = 1.0;
            for (int c = 0; c < D; ++c) {
              const int fa = c < d1 ? 0 : (c == d1 ? 1 : 2);
              const int fb = c < e1 ? 0 : (c == e1 ? 1 : 2);
              prod *= s_dots[c * 6 + idx[fa][fb]];
            }
            num += prod;
          }
        amp = 1.0;
        for (int c = 0; c < D; ++c) {
          den *= s_dots[c * 6 + 5];
          norms2[c] = s_dots[c * 6 + 5];
          amp *= s_max[c];
        }
        delta = den > 0.0 ? sqrt(fmax(num, 0.0) / den) : 0.0;
        __syncthreads();
      }
      if (P.fixed_als == 0 && delta <= P.tol_als) break;
      // Stall rule (optional): the change of the mode in units of the step's leading mode
      // (delta * amp against amp_lead; delta alone for the leading mode) is below als_stall
      // and no longer shrinking.  The mode has not met tol_als; it is counted as stalled.
      if (P.als_stall > 0.0 && P.fixed_als == 0 && it >= 3) {
        const double amp_lead = m == 0 ? amp : amp0;
        if (delta * amp <= P.als_stall * amp_lead && delta >= 0.5 * delta_prev) {
          ++n_stalled;
          break;
        }
      }
      delta_prev = delta;
    }
    if (it > n_it) it = n_it;
    if (m == 0) amp0 = amp;
    sweeps_max = max(sweeps_max, it);
    if (!zero_mode && P.fixed_als == 0 && !(delta <= P.tol_als)) not_conv = 1;
    if (zero_mode) amp = 0.0;
    if (P.fixed_modes == 0 && amp <= P.tol_enrich) { stopped = true; sweeps_discarded = it; break; }
    if (zero_mode) { stopped = true; sweeps_discarded = it; break; }   // fixed-mode runs cannot commit a zero mode
    // commit with equal 2-norms in every factor
    double scale[kMaxDim], target = 1.0;
    for (int c = 0; c < D; ++c) target *= sqrt(norms2[c]);
    target = pow(target, 1.0 / D);
    for (int c = 0; c < D; ++c) scale[c] = target / sqrt(norms2[c]);
    commit_mode(P, X, M, cb, scale);
    ++M;
    if (!sync_all(P, epoch, 7)) return;
    trace_mark(P, tmark, kTrCommit);
  }
  // ---- epilogue
  if (P.vrank == 0 && threadIdx.x == 0) {
    // adaptive CTD: M > M_c discards the separated result; u^k stays for the host's full-grid
    // step, which replaces it
    const bool switched = P.actd_Mc > 0 && P.fixed_modes == 0 && M > P.actd_Mc;
    InstState s = st0;
    if (switched) {
      s.switched = 1;
    } else {
      s.Mk = M;
      s.bank = cb;
      s.grid = 0;
      s.switched = 0;
    }
    s.step = st0.step + 1;
    s.status = P.st->status;
    *P.st = s;
    StepStatsDev r;
    r.modes = M;
    r.als_sweeps = sweeps;
    r.als_sweeps_max = sweeps_max;
    r.capped = (P.fixed_modes == 0 && !stopped && !switched) ? 1 : 0;
    r.actd_switched = switched ? 1 : 0;
    r.not_converged = not_conv;
    r.status = 0;
    r.als_stalled = n_stalled;
    r.als_sweeps_committed = sweeps - sweeps_discarded;
    r.cube_form = cube ? 1 : 0;
    *P.stats = r;
  }
}

static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
}

#ifdef CTD_SEPARATED_TU
// Time step with the separated nonlinear term (Eq. MxySep): no tensor-core or grid pass.
__global__ void __launch_bounds__(kThreads, 1) step_kernel_sep(const __grid_constant__ StepParams P,
                                                               const __grid_constant__ Extra X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepParams sP;
  __shared__ __align__(16) Extra sX;
  stage_params(&sP, P, gridDim.x, blockIdx.x);
  stage_to_smem(&sX, X);
  __syncthreads();
  step_body(sP, sX, smem_raw, 0u);
}

cudaError_t launch_step_sep(const StepParams& P, const Extra& X, int grid, cudaStream_t s) {
  const size_t smem = P.smem_bytes;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&step_kernel_sep), smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<StepParams*>(&P), const_cast<Extra*>(&X)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&step_kernel_sep), dim3(grid), dim3(kThreads),
                                     args, smem, s);
}
#else
__global__ void __launch_bounds__(kThreads, 1) step_kernel(const __grid_constant__ StepParams P,
                                                           const __grid_constant__ Extra X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(16) StepParams sP;
  __shared__ __align__(16) Extra sX;
  stage_params(&sP, P, gridDim.x, blockIdx.x);
  stage_to_smem(&sX, X);
  const bool tc = P.precision != 0;
  if (tc && (threadIdx.x >> 5) == 1) tmem_alloc(&s_tmem, kTcAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  step_body(sP, sX, smem_raw, tc ? s_tmem : 0u);
  __syncthreads();
  if (tc && (threadIdx.x >> 5) == 1) {
    tc_fence_after();
    tmem_dealloc(s_tmem, kTcAccCols);
  }
}

// Batched time steps: one CTA advances one instance (its own parameters and workspace,
// read from entries[order[blockIdx.x]]), with CTA-wide barriers in place of
// grid-wide ones.  kstep selects the instance's step record.  No CTA waits on another, so a
// plain launch with more instances than SMs is fine.
__global__ void __launch_bounds__(kThreads, 1) batch_step_kernel(const BatchEntry* entries, const int* order,
                                                                 int kstep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(16) StepParams sP;
  __shared__ __align__(16) Extra sX;
  const BatchEntry& E = entries[order[blockIdx.x]];
  stage_params(&sP, E.P, 1, 0);
  stage_to_smem(&sX, E.X);
  if (threadIdx.x == 0) sP.stats = E.P.stats + kstep;
  const bool tc = E.P.precision != 0;
  if (tc && (threadIdx.x >> 5) == 1) tmem_alloc(&s_tmem, kTcAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  step_body(sP, sX, smem_raw, tc ? s_tmem : 0u);
  __syncthreads();
  if (tc && (threadIdx.x >> 5) == 1) {
    tc_fence_after();
    tmem_dealloc(s_tmem, kTcAccCols);
  }
}

// ---------------------------------------------------------------------------------------
// Energy: bulk part sum_grid (prod omega) a0 (u^2 - 1)^2 with u rebuilt in FP64, per-CTA
// partial sums (fixed order); gradient part from the factors' Gram matrices.
__global__ void __launch_bounds__(kThreads) energy_bulk_kernel(const StepParams P, const Extra X, int Mk,
                                                               double* part) {
  const int D = P.dim;
  const int n0 = P.d[0].nq, n1 = P.d[1].nq, n2 = D == 3 ? P.d[2].nq : 1;
  const long long N = static_cast<long long>(n0) * n1 * n2;
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  double acc = 0.0;
  for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < N; p += stride) {
    double u = 0.0, w;
    if (P.quad) {
      // Gauss rule: u^k at the Gauss points from the factors there, weights omega_q
      const int l = static_cast<int>(p % n2);
      const long long ij = p / n2;
      const int j = static_cast<int>(ij % n1), i = static_cast<int>(ij / n1);
      for (int m = 0; m < Mk; ++m) {
        double t = f2_to_double(P.d[0].Aq[static_cast<size_t>(m) * n0 + i]) *
                   f2_to_double(P.d[1].Aq[static_cast<size_t>(m) * n1 + j]);
        if (D == 3) t *= f2_to_double(P.d[2].Aq[static_cast<size_t>(m) * n2 + l]);
        u += t;
      }
      w = P.d[0].wq[i] * P.d[1].wq[j] * (D == 3 ? P.d[2].wq[l] : 1.0);
    } else if (D == 2) {
      const int i = static_cast<int>(p / n1), j = static_cast<int>(p - static_cast<long long>(i) * n1);
      for (int m = 0; m < Mk; ++m)
        u = fma(X.Af[0][static_cast<size_t>(m) * n0 + i], X.Af[1][static_cast<size_t>(m) * n1 + j], u);
      w = P.d[0].omega[i] * P.d[1].omega[j];
    } else {
      const int l = static_cast<int>(p % n2);
      const long long ij = p / n2;
      const int j = static_cast<int>(ij % n1), i = static_cast<int>(ij / n1);
      for (int m = 0; m < Mk; ++m)
        u = fma(X.Af[0][static_cast<size_t>(m) * n0 + i] * X.Af[1][static_cast<size_t>(m) * n1 + j],
                X.Af[2][static_cast<size_t>(m) * n2 + l], u);
      w = P.d[0].omega[i] * P.d[1].omega[j] * P.d[2].omega[l];
    }
    const double t = u * u - 1.0;
    acc = fma(w * P.a0, t * t, acc);
  }
  acc = warp_sum(acc);
  __shared__ double s[kWarps];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += s[w];
    part[blockIdx.x] = t;
  }
}

// Gauss rule: the current factors at the Gauss points (whole arrays, double-float)
__global__ void gauss_points_kernel(const StepParams P, int bank, int Mk) {
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    const long long total = static_cast<long long>(Mk) * dd.nq;
    for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<long long>(gridDim.x) * blockDim.x) {
      const int m = static_cast<int>(t / dd.nq), r = static_cast<int>(t - static_cast<long long>(m) * dd.nq);
      const dfloat v = phi_row(dd, dd.b + 1, dd.bank[bank] + static_cast<size_t>(m) * dd.n, r);
      dd.Aq[t] = make_float2(v.hi, v.lo);
    }
  }
}

// FP64 copies of the current factors (whole arrays)
__global__ void convert_modes_kernel(const StepParams P, const Extra X, int bank, int Mk) {
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    const long long total = static_cast<long long>(Mk) * dd.n;
    for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<long long>(gridDim.x) * blockDim.x)
      X.Af[d][t] = f2_to_double(dd.bank[bank][t]);
  }
}

// Gram matrices of the current factors: out[d][2][Mk][Mk] = (b^T M b', b^T K b') in FP64
__global__ void energy_gram_kernel(const StepParams P, const Extra X, int Mk, double* out) {
  const int d = blockIdx.y;
  const Dim& dd = P.d[d];
  const int pair = blockIdx.x;
  const int m1 = pair / Mk, m2 = pair % Mk;
  const double* a = X.Af[d] + static_cast<size_t>(m1) * dd.n;
  const double* c = X.Af[d] + static_cast<size_t>(m2) * dd.n;
  double sm = 0.0, sk = 0.0;
  const int w = 2 * dd.b + 1;
  for (int i = threadIdx.x; i < dd.n; i += blockDim.x) {
    if (dd.mband) {   // Gauss rule: consistent mass band
      double mc = 0.0;
      for (int j = max(0, i - dd.b); j <= min(dd.n - 1, i + dd.b); ++j)
        mc = fma(dd.mband[static_cast<size_t>(i) * w + (j - i + dd.b)], c[j], mc);
      sm = fma(a[i], mc, sm);
    } else {
      sm = fma(a[i] * dd.omega[i], c[i], sm);
    }
    double kc = 0.0;
    for (int j = max(0, i - dd.b); j <= min(dd.n - 1, i + dd.b); ++j)
      kc = fma(dd.kband[static_cast<size_t>(i) * w + (j - i + dd.b)], c[j], kc);
    sk = fma(a[i], kc, sk);
  }
  sm = warp_sum(sm);
  sk = warp_sum(sk);
  __shared__ double s[2][kWarps];
  if ((threadIdx.x & 31) == 0) { s[0][threadIdx.x >> 5] = sm; s[1][threadIdx.x >> 5] = sk; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int k = 0; k < kWarps; ++k) { t0 += s[0][k]; t1 += s[1][k]; }
    out[(static_cast<size_t>(d) * 2 + 0) * Mk * Mk + pair] = t0;
    out[(static_cast<size_t>(d) * 2 + 1) * Mk * Mk + pair] = t1;
  }
}

// ---------------------------------------------------------------------------------------
// Probe kernels
__device__ void probe_contract_body(const StepParams& P, const Extra& X, int x, float* dump,
                                    unsigned char* smem_raw, uint32_t tmem_base) {
  const Arena ar = arena_of(smem_raw, P);
  unsigned epoch = 0;
  const InstState st0 = *P.st;
  if (P.precision == 0) {
    convert_prev_modes(P, X, st0.bank, st0.Mk);
    if (P.quad) gauss_prologue(P, X, st0.bank, st0.Mk);
    if (!sync_all(P, epoch, 11)) return;
    if (P.quad) materialise_w_gauss(P, st0.Mk);
    else materialise_w(P, X, st0.Mk);
    if (!sync_all(P, epoch, 12)) return;
    GridW g;
    if (P.quad) {
      g = load_weights_gauss(P, x, ar.wv);
    } else {
      load_weights_fp64(P, X, x, ar.wv);
      g = nodal_grid(P, ar.wv);
    }
    contract_fp64(P, x, g);
  } else {
    if (P.quad) {
      gauss_prologue(P, X, st0.bank, st0.Mk);
      if (!sync_all(P, epoch, 13)) return;
    }
    // the step's choice of contraction form (the dump is of u: direct form)
    const int Mk = st0.Mk, pb = st0.bank;
    float* fs = reinterpret_cast<float*>(arena_base(smem_raw));
    bool cube = false;
    if (!dump && Mk > 0 && P.reduced_tol <= 0.0 && P.contraction_form != 1)
      cube = P.contraction_form == 2 || tc_amp_bound(P, pb, Mk, fs) <= kCubeMaxAmp;
    tc_prepare(P, X.dirs, X.kr, pb, Mk, !cube);
    const TcDir& td = X.dirs[x];
    if (cube) tc_prepare_scaled(P, X.kc, td, X.kr[x], pb, Mk, fs);
    fence_proxy_async_global();
    if (!sync_all(P, epoch, 11)) return;
    const __nv_bfloat16* qop = (P.dim == 2 && !cube) ? P.d[td.last].op : X.kr[x];
    tc_contract(P, X.kc, td, P.d[x].op, qop, x, Mk, X.tc_stages, arena_base(smem_raw), tmem_base, X.rpart_tc,
                dump, nullptr, 0.f, 0.f, cube);
    if (P.vrank == 0 && threadIdx.x == 0) X.ctrl[2] = cube ? 1 : 0;
    if (!cube) return;
    // the cube form's linear part for the host, lin_i = sum_m A_m,i H_m into P.rpart (A the
    // factors, or M a under the Gauss rule; H_m the product over the other dimensions of
    // h_d,m = sum_j omega_j v_j a_m(j), or v . M a_m): FP64, every CTA forms H alike
    double* sH = reinterpret_cast<double*>(arena_base(smem_raw));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nO = P.dim - 1;
    __syncthreads();
    for (int t = warp; t < nO * Mk; t += kWarps) {
      const int o = t / Mk, m = t - o * Mk, d = o < x ? o : o + 1;
      const Dim& dd = P.d[d];
      const float2* a = (P.quad ? dd.MA : dd.bank[pb]) + static_cast<size_t>(m) * dd.n;
      double acc = 0.0;
      for (int j = lane; j < dd.n; j += 32) {
        const float2 vv = dd.v[j], aa = a[j];
        const double w = P.quad ? 1.0 : dd.omega[j];
        acc = fma(w * (static_cast<double>(vv.x) + vv.y), static_cast<double>(aa.x) + aa.y, acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) sH[t] = acc;
    }
    __syncthreads();
    const Dim& dx = P.d[x];
    const float2* A = P.quad ? dx.MA : dx.bank[pb];
    for (int i = P.vrank * blockDim.x + threadIdx.x; i < dx.n; i += P.vgrid * blockDim.x) {
      double lin = 0.0;
      for (int m = 0; m < Mk; ++m) {
        double H = 1.0;
        for (int o = 0; o < nO; ++o) H *= sH[o * Mk + m];
        const float2 am = A[static_cast<size_t>(m) * dx.n + i];
        lin = fma(static_cast<double>(am.x) + am.y, H, lin);
      }
      P.rpart[i] = lin;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) probe_contract_kernel(const __grid_constant__ StepParams P,
                                                                     const __grid_constant__ Extra X,
                                                                     int x,
                                                                     float* dump) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(16) StepParams sP;
  __shared__ __align__(16) Extra sX;
  stage_params(&sP, P, gridDim.x, blockIdx.x);
  stage_to_smem(&sX, X);
  const bool tc = P.precision != 0;
  if (tc && (threadIdx.x >> 5) == 1) tmem_alloc(&s_tmem, kTcAccCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  probe_contract_body(sP, sX, x, dump, smem_raw, tc ? s_tmem : 0u);
  __syncthreads();
  if (tc && (threadIdx.x >> 5) == 1) {
    tc_fence_after();
    tmem_dealloc(s_tmem, kTcAccCols);
  }
}

__global__ void __launch_bounds__(kThreads, 1) probe_solve_kernel(const __grid_constant__ StepParams Pp,
                                                                  const __grid_constant__ Extra Xp, int x,
                                                                  double a1, double a2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) StepParams P;
  __shared__ __align__(16) Extra X;
  stage_params(&P, Pp, 1, 0);
  stage_to_smem(&X, Xp);
  __syncthreads();
  SmemStep& sm = *reinterpret_cast<SmemStep*>(smem_raw);
  const Arena ar = arena_of(smem_raw, P);
  if (threadIdx.x == 0) {
    st_df(&sm.coef.alpha1, df_of(a1));
    st_df(&sm.coef.alpha2, df_of(a2));
  }
  __syncthreads();
  const Dim& dd = P.d[x];
  const SolverStore ss = solver_bind(P.solver_mode == 2 ? 0 : P.solver_mode, ar.solver, P.solver, dd.n, dd.b, dd.mu_max);
  bool ok = banded_solve(ss, X.kc[x], ld_df(&sm.coef.alpha1), ld_df(&sm.coef.alpha2), P.Q, ar.xsol, sm.redf, P.trace);
  for (int i = threadIdx.x; i < dd.n; i += blockDim.x) dd.v[i] = ar.xsol[i];
  if (threadIdx.x == 0) X.ctrl[1] = ok ? 0 : 1;
}

size_t step_smem_fixed_bytes() { return kArenaOffset; }
size_t step_arena_bytes(int n_max, size_t solver_floats, int mode) {
  size_t c;
  if (mode == 0 || mode == 3) c = solver_smem_offset(n_max) + solver_floats * sizeof(float);
  else if (mode == 1) c = solver_floats * sizeof(float);
  else c = solver_smem_offset(n_max);
  return std::max(arena_phase_a_bytes(), c);
}

}  // namespace ctd

namespace ctd {

__global__ void f64_to_df_kernel(float2* dst, const double* src, long long count) {
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < count;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const dfloat v = df_from_double(src[t]);
    dst[t] = make_float2(v.hi, v.lo);
  }
}
__global__ void df_to_f64_kernel(double* dst, const float2* src, long long count) {
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < count;
       t += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[t] = f2_to_double(src[t]);
}


cudaError_t launch_step(const StepParams& P, const Extra& X, int grid, cudaStream_t s) {
  const size_t smem = P.smem_bytes;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&step_kernel), smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<StepParams*>(&P), const_cast<Extra*>(&X)};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&step_kernel), dim3(grid), dim3(kThreads),
                                     args, smem, s);
}

cudaError_t launch_batch_step(const BatchEntry* entries, const int* order, int count, int kstep, size_t smem,
                              cudaStream_t s) {
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&batch_step_kernel), smem);
  if (e != cudaSuccess) return e;
  batch_step_kernel<<<count, kThreads, smem, s>>>(entries, order, kstep);
  return cudaGetLastError();
}

cudaError_t launch_probe_contract(const StepParams& P, const Extra& X, int grid, int x,
                                  float* dump, cudaStream_t s) {
  const size_t smem = P.smem_bytes;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&probe_contract_kernel), smem);
  if (e != cudaSuccess) return e;
  void* args[] = {const_cast<StepParams*>(&P), const_cast<Extra*>(&X), &x, &dump};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&probe_contract_kernel), dim3(grid),
                                     dim3(kThreads), args, smem, s);
}

cudaError_t launch_probe_solve(const StepParams& P, const Extra& X, int x, double a1, double a2,
                               cudaStream_t s) {
  const size_t smem = P.smem_bytes;
  cudaError_t e = set_smem(reinterpret_cast<const void*>(&probe_solve_kernel), smem);
  if (e != cudaSuccess) return e;
  probe_solve_kernel<<<1, kThreads, smem, s>>>(P, X, x, a1, a2);
  return cudaGetLastError();
}

cudaError_t launch_convert_modes(const StepParams& P, const Extra& X, int bank, int Mk, cudaStream_t s) {
  convert_modes_kernel<<<256, kThreads, 0, s>>>(P, X, bank, Mk);
  if (P.quad && Mk > 0) gauss_points_kernel<<<256, kThreads, 0, s>>>(P, bank, Mk);
  return cudaGetLastError();
}

cudaError_t launch_energy_bulk(const StepParams& P, const Extra& X, int Mk, double* part, int grid,
                               cudaStream_t s) {
  energy_bulk_kernel<<<grid, kThreads, 0, s>>>(P, X, Mk, part);
  return cudaGetLastError();
}

cudaError_t launch_energy_gram(const StepParams& P, const Extra& X, int Mk, double* out, cudaStream_t s) {
  if (Mk == 0) return cudaSuccess;
  energy_gram_kernel<<<dim3(Mk * Mk, P.dim), kThreads, 0, s>>>(P, X, Mk, out);
  return cudaGetLastError();
}

cudaError_t launch_modes_from_fp64(float2* dst, const double* src, long long count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  f64_to_df_kernel<<<256, kThreads, 0, s>>>(dst, src, count);
  return cudaGetLastError();
}

cudaError_t launch_modes_to_fp64(double* dst, const float2* src, long long count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  df_to_f64_kernel<<<256, kThreads, 0, s>>>(dst, src, count);
  return cudaGetLastError();
}

#endif  // CTD_SEPARATED_TU
}  // namespace ctd

// Shared device-side definitions of the CTD step: parameter blocks, the bounded grid
// barrier, double-float (two FP32 words) arithmetic and the SplitMix64 generator.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ctd {

constexpr int kThreads = 256;          // threads per CTA of the step kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxDim = 3;
constexpr int kMaxN = 4096;            // nodes per dimension
constexpr int kMaxModes = 128;         // M_max limit
// Separated nonlinearity: u^3 of a rank-M_k field has one separated term per multiset
// {m1 <= m2 <= m3} of mode indices; used for M_k up to kMaxSepModes (kMaxSep multisets)
constexpr int kMaxSepModes = 16;
constexpr int kMaxSep = kMaxSepModes * (kMaxSepModes + 1) * (kMaxSepModes + 2) / 6;
__host__ __device__ constexpr int sep_terms(int Mk) { return Mk * (Mk + 1) * (Mk + 2) / 6; }
constexpr int kTileRows = 128;         // tensor-core tile rows (operand rows padded to this)
constexpr int kPhiW = 8;               // shape functions nonzero on one element: 2s + 2 <= 8

// status bits written by the kernels (host maps them to ctd_status)
constexpr int kErrTimeout = 1;
constexpr int kErrNonfinite = 2;
constexpr int kErrSolve = 4;

struct Dim {
  int n;                   // nodes
  int b;                   // half bandwidth of K (2s+1)
  int n_pad;               // rows padded to kTileRows (tensor-core operands)
  const double* omega;     // [n] nodal weights (FP64)
  const double* kband;     // [n][2b+1] stiffness band (FP64)
  float2* bank[2];         // [Mcap][n] factor banks (double-float): u^k and u^{k+1} alternate
  float2* KB;              // [Mcap][n] K * committed factors of the step being built
  float2* v;               // [n] trial factor (double-float)
  float2* vold;            // [n] trial factor at the start of the sweep
  __nv_bfloat16* op;       // [n_pad][2*Kpad] tensor-core operand: hi | lo split of u^k
  float mu_max;            // Gershgorin bound of the generalised eigenvalues of (K, diag(omega))
  // Quadrature points of the mass-type integrals: the nodes (nodal rule, nq = n) or q Gauss
  // points per element (Gauss rule, nq = q (n - 1)); the grid of the nonlinear term is the
  // tensor product of the points.  Gauss rule only (null otherwise):
  int nq;                  // points
  const double* wq;        // [nq] weights
  const float2* phi;       // [nq][kPhiW] shape function values N~_{phi0[r]+k}(x_r) (double-float)
  const int* phi0;         // [nq] first node of each point's shape function row
  const double* mband;     // [n][2b+1] consistent mass band (FP64)
  float2* MA;              // [Mcap][n] M a of u^k's factors (double-float)
  float2* MB;              // [Mcap][n] M b of u^{k+1}'s committed factors (double-float)
  float2* Aq;              // [Mcap][nq] Phi a: u^k's factors at the points (double-float)
};

struct InstState {
  int Mk;                  // number of modes of u^k
  int bank;                // bank index holding u^k
  long long step;          // index of the next step (SplitMix64 key)
  int status;              // kErr* bits
  int err_info;            // where a wait gave up (phase id)
  int grid;                // 1: u^k is held as the full-grid array U (after an adaptive-CTD step)
  int switched;            // 1: the last step reached M_c + 1 modes; the host solves it on the grid
};

struct StepStatsDev {
  int modes;
  int als_sweeps;
  int als_sweeps_max;
  int capped;
  int not_converged;
  int status;
  int als_stalled;
  int als_sweeps_committed;
  int actd_switched;
  int cube_form;
};

struct StepParams {
  int dim;
  Dim d[kMaxDim];
  int Mcap;                // columns per bank
  int Kpad;                // padded mode count of the tensor-core operands (multiple of 64)
  int precision;           // 0 FP64, 1 split BF16 tensor cores
  int quad;                // 0 nodal rule (M = diag(omega)), 1 Gauss rule (consistent mass)
  int actd_Mc;             // > 0: adaptive CTD critical mode count (budget M_c + 1)
  double* U;               // [N] full-grid field of the adaptive-CTD grid state (FP64)
  int quad_q;              // Gauss points per element
  double c_t, c_k, L, a0;
  float2 ct_df, ck_df, L_df;   // the same constants as double-float (converted on the host)
  double tol_als, tol_enrich;
  double als_stall;        // > 0: stall rule of the fixed-point sweeps (0: off)
  int I_max, M_max, fixed_als, fixed_modes;
  unsigned long long seed;
  unsigned long long wait_ns;
  // workspace scratch
  double* W;               // [N] w(u^k) on the grid (FP64 path)
  float2* gram;            // [slots][grid] per-CTA partial sums (double-float), slot-major
  double* rpart;           // [n_x][rchunks[x]] partial contractions
  int rchunks[kMaxDim];
  float2* Q;               // [kMaxN] right-hand side (double-float)
  float* solver;           // CR factor storage for the solver CTA
  unsigned* barrier;       // grid barrier counter (zeroed before each launch)
  InstState* st;
  StepStatsDev* stats;     // one record per launch
  unsigned long long* trace;   // null, or [kTraceSlots] ns accumulated per phase by CTA 0
  int solver_mode;         // 0: full CR factors in shared memory; 1: first level on the fly,
                           // level-1 factors in shared memory; 2: full CR factors in global;
                           // 3: Chebyshev semi-iteration, vectors in shared memory
  float2* xsol_g;          // [kMaxN] solution iterate in global memory (solver mode 1)
  int smem_bytes;          // dynamic shared memory of the step kernel
  int n_max;               // largest n over the dimensions
  double reduced_tol;      // > 0: reduced integration domain of the nonlinear term (2D)
  unsigned* tile_max;      // [nrb_0 * ntc_0] max |u(u^2-1)| per 128 x 128 node block (float bits)
  int nl_form;             // 0: nonlinear term as the full nodal integral (Eq. KxxMxx); 1: the
                           // separated form (Eq. MxySep) for steps with M_k <= kMaxSepModes
  int sep_q;               // Gram slots per dimension reserved for the separated form (0 if off)
  int contraction_form;    // tensor-core epilogue: 0 automatic, 1 direct, 2 cube (see ctd_contract_tc.cuh)
  int vgrid, vrank;        // CTAs working on this instance and this CTA's rank among them: the
                           // launch grid for a single instance, 1 and 0 in a batched launch
                           // (set by each CTA in its shared-memory copy)
};

// phases accumulated in StepParams::trace (each includes its closing grid barrier)
enum TracePhase { kTrPrologue = 0, kTrInit, kTrGramContract, kTrRhs, kTrSolve, kTrConverge, kTrCommit,
                  kTrScale,   // the cube form's scaled column operand (per half-sweep)
                  kTrSolveFactor = 8, kTrSolveFirst, kTrSolveRefine, kTrSolvePasses, kTrGram, kTrContract,
                  kTrSolveResidual, kTrSolveInner,
                  // tensor-core contraction roles on the traced CTA, SM clock cycles: producer waiting
                  // for a free stage, MMA issuer waiting for operands / for a free accumulator and
                  // issuing, epilogue waiting for an accumulator and working, tiles contracted
                  kTrTcProdWait = 16, kTrTcMmaWaitB, kTrTcMmaWaitAcc, kTrTcMmaIssue, kTrTcEpiWait, kTrTcEpiWork,
                  kTrTcTiles, kTrSlots = 24 };

// ------------------------------------------------------------------ time & barrier
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier over all CTAs of a (co-resident) launch.  The counter only grows
// within a launch: barrier number k completes when it reaches (k+1) * gridDim.x.  Thread 0
// arrives with a release reduction and polls with acquire loads; the wait gives up after
// wait_ns, sets kErrTimeout and returns false (the caller then leaves the kernel).
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned& epoch,
                                             unsigned long long wait_ns, InstState* st,
                                             int where) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1;
    const unsigned target = epoch * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(counter) : "memory");
    unsigned v;
    int ok = 1;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
    if (static_cast<int>(v - target) < 0) {
      // waiting: also watch the instance status, so that a CTA that timed out elsewhere makes
      // the others fail fast (checked only while waiting: no extra load on the fast path)
      const unsigned long long t0 = global_ns();
      while (true) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
        if (static_cast<int>(v - target) >= 0) break;
        if (*reinterpret_cast<volatile int*>(&st->status) & kErrTimeout) {
          ok = 0;
          break;
        }
        if (global_ns() - t0 > wait_ns) {
          ok = 0;
          atomicOr(&st->status, kErrTimeout);
          atomicExch(&st->err_info, where);
          break;
        }
      }
    }
    s_ok = ok;
  } else {
    epoch += 1;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------ double-float
// A value is hi + lo with |lo| <= ulp(hi)/2 (about 48 significant bits).  Error-free
// transformations after Knuth (TwoSum) and Dekker (TwoProduct with a fused multiply-add).
struct dfloat { float hi, lo; };

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  dfloat s = df_two_sum(a.hi, b.hi);
  dfloat t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = df_fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return df_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a + b * c
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat b, dfloat c) {
  return df_add(a, df_mul(b, c));
}
__device__ __forceinline__ dfloat df_from_double(double x) {
  const float hi = __double2float_rn(x);
  const float lo = __double2float_rn(x - static_cast<double>(hi));
  return {hi, lo};
}
__device__ __forceinline__ double df_to_double(dfloat a) {
  return static_cast<double>(a.hi) + static_cast<double>(a.lo);
}
__device__ __forceinline__ double f2_to_double(float2 a) {
  return static_cast<double>(a.x) + static_cast<double>(a.y);
}

// ------------------------------------------------------------------ SplitMix64
// Steele, Lea & Flood (OOPSLA 2014) output function applied to x + golden gamma.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Start vector of a mode without a warm start: chained key (seed, step, 4*mode+dim, node),
// 53 random bits to [0, 1), shifted to [0.5, 1.5).
__device__ __forceinline__ double mode_init_value(unsigned long long seed, long long step,
                                                  int mode, int dim, int node) {
  unsigned long long h = splitmix64(seed);
  h = splitmix64(h ^ static_cast<unsigned long long>(step));
  h = splitmix64(h ^ static_cast<unsigned long long>(4 * mode + dim));
  h = splitmix64(h ^ static_cast<unsigned long long>(node));
  return 0.5 + static_cast<double>(h >> 11) * (1.0 / 9007199254740992.0);
}

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// contiguous slice [lo, hi) of n items owned by part `k` of `parts`
__device__ __forceinline__ void slice_of(int n, int parts, int k, int& lo, int& hi) {
  const long long a = static_cast<long long>(n) * k / parts;
  const long long b = static_cast<long long>(n) * (k + 1) / parts;
  lo = static_cast<int>(a);
  hi = static_cast<int>(b);
}

}  // namespace ctd

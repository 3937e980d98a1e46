// Nonlinear contraction of Eq. KxxMxx on the 5th-generation tensor cores (sm_103a).
//
// For direction x, with P the factors of u^k in dimension x (n_x x M_k) and Q the factors of
// the other dimension (2D) or their row-wise (Khatri-Rao) products (3D), the grid values
// of u^k are U = P Q^T.  Each CTA walks a contiguous range of 128 x 128 tiles of U:
//   * the operands are stored as tile images: per 128-row block and 16-wide K step a hi and a
//     lo image of 128 x 16 BF16 in the canonical K-major layout without swizzle, so that one
//     bulk TMA copy (cp.async.bulk) brings a row block's K steps into shared memory: P's
//     block once per row block, Q's column blocks through a ring of stages;
//   * one thread issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate in TMEM) for the
//     split product U = P_hi Q_hi^T + P_hi Q_lo^T + P_lo Q_hi^T (P = P_hi + P_lo in BF16);
//   * four epilogue warps read the accumulator rows with tcgen05.ld and fuse the cubic
//     w(u)/(4 a0) = u (u^2 - 1) with the weighted row sum over the tile's columns (weights
//     4 a0 omega v of the fixed factors), accumulating per row in FP32;
//   * four TMEM accumulators rotate so the MMAs of the next tiles overlap the epilogue of t.
// Every wait is bounded in time; on expiry the kernel records kErrTimeout and unwinds.
#pragma once

#include "ctd_common.cuh"
#include "ctd_solve.cuh"

namespace ctd {

constexpr int kTcN = 128;              // columns per tile (UMMA N)
constexpr int kTcM = 128;              // rows per tile (UMMA M)
// Shared-memory sizing unit: a row block's image of 2 Kpad K columns (hi and lo) takes
// (2 Kpad / kTcChunkElems) units of kTcChunkBytes
constexpr int kTcChunkElems = 64;
constexpr int kTcChunkBytes = kTcM * 128;   // 16 KB
constexpr int kTcAcc = 4;              // TMEM accumulators in flight (MMAs run ahead of the epilogue)
constexpr int kTcAccCols = kTcAcc * kTcN;   // TMEM columns allocated: all 512 of the SM

// Tile-image operand layout.  Rows come in blocks of 128; a block holds KS = Kpad / 16 K steps,
// each `nimg` images of 4 KB (the BF16 terms of the split: hi, or hi and lo, or hi, mid and
// lo): 16 groups of 8 rows (256 bytes apart), each group two core matrices of 8 rows x 8
// columns (128 contiguous bytes, the second holding columns 8..15).
constexpr int kTcImgElems = kTcM * 16;                  // elements of one image
constexpr uint32_t kTcImgBytes = kTcImgElems * 2;       // 4 KB
__host__ __device__ inline size_t tc_img_index(long long i, int k, int h, int KS, int nimg) {
  const long long rb = i >> 7;
  const int r = static_cast<int>(i & 127), g = r >> 3, rr = r & 7;
  const int ks = k >> 4, j = (k >> 3) & 1, e = k & 7;
  return static_cast<size_t>(((rb * KS + ks) * nimg + h) * kTcImgElems) + g * 128 + j * 64 + rr * 8 + e;
}
// BF16 terms per operand value for a tensor-core precision (1: BF16, 2: hi + lo, 3: hi + mid +
// lo) and the products the reconstruction sums: every pair (a, b) of terms of order below the
// last term's, i.e. all a + b <= nimg - 1 (1, 3 or 6 MMAs per K step).
__host__ __device__ constexpr int tc_nimg(int precision) { return precision == 2 ? 1 : (precision == 3 ? 3 : 2); }
__host__ __device__ constexpr int tc_npairs(int nimg) { return nimg * (nimg + 1) / 2; }
// product p: terms (tc_pair_a(p), tc_pair_b(p)) in the order (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
__host__ __device__ constexpr int tc_pair_a(int p) { return (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0); }
__host__ __device__ constexpr int tc_pair_b(int p) { return (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0); }

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false (and kErrTimeout recorded) on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns,
                                          InstState* st, const volatile int* abort_flag, int where) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 > limit_ns) {
      atomicOr(&st->status, kErrTimeout);
      atomicExch(&st->err_info, where);
      return false;
    }
  }
}
// The same wait by every lane of a warp; the warp leaves it converged and agreeing on the result
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, unsigned long long limit_ns, InstState* st,
                                          const volatile int* abort_flag, int where) {
  const bool r = mbar_wait(bar, parity, limit_ns, st, abort_flag, where);
  return __all_sync(0xffffffffu, r);
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Generic-proxy global writes (operand preparation) made visible to later TMA reads
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Bulk TMA copy global -> shared (both 16-byte aligned, bytes a multiple of 16), completion
// counted on the mbarrier's transaction bytes
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulator
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  // The load writes r[] asynchronously, when the wait completes: r[] pass through the wait
  // as read-write operands, so that the compiler neither reads them before it nor reuses
  // their registers in between (a late write would clobber whatever it put there).
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of one tile image: K-major, no swizzle, core matrices
// adjacent in K 128 bytes apart (leading byte offset), 8-row groups 256 bytes apart (stride
// byte offset).
__device__ __forceinline__ uint64_t umma_desc_img(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFF) >> 4);   // start address
  d |= static_cast<uint64_t>(128 >> 4) << 16;           // leading byte offset
  d |= static_cast<uint64_t>(256 >> 4) << 32;           // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version
  return d;                                             // swizzle mode 0: none
}
// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = kTcN.
__host__ __device__ constexpr uint32_t umma_idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(kTcN >> 3) << 17) |
         (static_cast<uint32_t>(kTcM >> 4) << 24);
}

// ---------------------------------------------------------------- tile schedule
struct TcPlan {
  int nrb;        // row blocks of direction x (n_pad_x / 128)
  int ntc;        // column tiles (n_cols_pad / 128)
  int ncols_pad;  // padded column count of the Q operand
  int chunks;     // 64-element K chunks per operand row (= 2 * Kpad / 64)
  int kpad;       // Kpad
  int ksteps;     // 16-wide K steps covering M_k
  int stages;     // B ring depth
  int cmax;       // partial slots per row
};

// The first kLightCtas CTAs also compute the Gram partial sums before their tiles; they take
// an eighth of the tiles of the others so that all finish together.  CTA c owns the contiguous
// tile range [tile_lo(c), tile_lo(c + 1)) with tile_lo(c) = floor(T cum(c) / tot), cum(c) the
// weight units before c (1 per light CTA, kHeavyWeight per other) and tot = cum(G).
constexpr int kLightCtas = 16;
constexpr int kHeavyWeight = 8;
__host__ __device__ inline long long tile_cum(int G, int c) {
  const int L = G < kLightCtas ? G : kLightCtas;
  return c <= L ? c : L + static_cast<long long>(kHeavyWeight) * (c - L);
}
// floor(a / b) for a, b >= 0; 32-bit division when both fit
__host__ __device__ inline long long tile_div(long long a, long long b) {
  if (a < 0xFFFFFFFFLL) return static_cast<long long>(static_cast<unsigned>(a) / static_cast<unsigned>(b));
  return a / b;
}
__host__ __device__ inline int tile_lo(long long T, int G, int c) {
  return static_cast<int>(tile_div(T * tile_cum(G, c), tile_cum(G, G)));
}
// CTA that owns tile t (0 <= t < T): the largest c < G with tile_lo(c) <= t, i.e. with
// cum(c) <= kmax = floor(((t + 1) tot - 1) / T)
__host__ __device__ inline int tile_owner(long long T, int G, long long t) {
  const int L = G < kLightCtas ? G : kLightCtas;
  const long long kmax = tile_div((t + 1) * tile_cum(G, G) - 1, T);
  const long long c = kmax <= L ? kmax : L + (kmax - L) / kHeavyWeight;
  return static_cast<int>(c < G - 1 ? c : G - 1);
}

struct TcShared {           // barriers and TMEM handle (placed at the start of the arena)
  uint64_t a_full, a_empty;
  uint64_t b_full[8], b_empty[8];
  uint64_t acc_full[kTcAcc], acc_empty[kTcAcc];
  uint32_t tmem_base;
  int abort;
};

}  // namespace ctd

namespace ctd {

// Per-direction geometry of the tensor-core contraction (filled on the host).
struct TcDir {
  int nrb;          // row blocks of direction x
  int ntc;          // column tiles
  int ncols_pad;    // padded rows of the column operand
  int n_last_pad;   // 3D: padded length of the last other dimension (tile = one mid index)
  int mid, last;    // other dimensions: 2D mid = -1, last = the other; 3D both set
  int cmax;         // partial slots per row in rpart_tc
};

// Split u^k's factors into BF16 hi/lo tile-image operands and, in 3D, the Khatri-Rao operands
// of the two other dimensions for every direction.  Only the K steps that hold modes are
// written.  One unit = 8 consecutive K columns of one row (one 16-byte core-matrix row of the
// hi and of the lo image); units in image order, grid-stride over all CTAs.
static __device__ __noinline__ void tc_prepare(const StepParams& P, const TcDir* dirs, __nv_bfloat16* const* kr, int pb,
                                  int Mk, bool build_kr = true) {
  const int KS = P.Kpad / 16, ksteps = (Mk + 15) / 16, nimg = tc_nimg(P.precision);
  const long long stride = static_cast<long long>(P.vgrid) * blockDim.x;
  const long long t0 = static_cast<long long>(P.vrank) * blockDim.x + threadIdx.x;
  // unit u -> (row block, K step, group, core matrix, row in group)
  auto unit = [&](long long u, long long& i, int& k0) {
    const int rr = static_cast<int>(u & 7), j = static_cast<int>((u >> 3) & 1), g = static_cast<int>((u >> 4) & 15);
    const long long q = u >> 8;
    const int ks = static_cast<int>(q % ksteps);
    i = (q / ksteps) * 128 + g * 8 + rr;
    k0 = ks * 16 + j * 8;
  };
  // the BF16 terms of the split: t_0 = bf16(a), t_h = bf16(a - t_0 - .. - t_{h-1}) (each
  // remainder is exact in FP32)
  auto store = [&](__nv_bfloat16* op, long long i, int k0, const float (&a)[8]) {
    float rem[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) rem[e] = a[e];
    const size_t o = tc_img_index(i, k0, 0, KS, nimg);
    for (int h = 0; h < nimg; ++h) {
      __align__(16) __nv_bfloat16 t[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        t[e] = __float2bfloat16_rn(rem[e]);
        rem[e] -= __bfloat162float(t[e]);
      }
      *reinterpret_cast<uint4*>(op + o + static_cast<size_t>(h) * kTcImgElems) = *reinterpret_cast<const uint4*>(t);
    }
  };
  if (ksteps == 0) return;
  // rows: the nodes (nodal rule, factors) or the Gauss points (Gauss rule, factors there)
  auto src_of = [&](const Dim& dd) { return P.quad ? dd.Aq : dd.bank[pb]; };
  for (int d = 0; d < P.dim; ++d) {
    const Dim& dd = P.d[d];
    const float2* src = src_of(dd);
    const int rows = dd.nq;
    const long long total = static_cast<long long>(dd.n_pad) * ksteps * 2;
    for (long long u = t0; u < total; u += stride) {
      long long i;
      int k0;
      unit(u, i, k0);
      float a[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        a[e] = 0.f;
        if (i < rows && k < Mk) {
          const float2 v = src[static_cast<size_t>(k) * rows + i];
          a[e] = v.x + v.y;
        }
      }
      store(dd.op, i, k0, a);
    }
  }
  if (P.dim != 3 || !build_kr) return;
  for (int x = 0; x < 3; ++x) {
    const TcDir& td = dirs[x];
    const Dim& dm = P.d[td.mid];
    const Dim& dl = P.d[td.last];
    const long long total = static_cast<long long>(td.ncols_pad) * ksteps * 2;
    for (long long u = t0; u < total; u += stride) {
      long long row;
      int k0;
      unit(u, row, k0);
      const int j = static_cast<int>(row / td.n_last_pad), l = static_cast<int>(row - static_cast<long long>(j) * td.n_last_pad);
      const float2* sm = src_of(dm);
      const float2* sl = src_of(dl);
      float a[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        a[e] = 0.f;
        if (j < dm.nq && l < dl.nq && k < Mk) {
          const float2 vm = sm[static_cast<size_t>(k) * dm.nq + j];
          const float2 vl = sl[static_cast<size_t>(k) * dl.nq + l];
          a[e] = (vm.x + vm.y) * (vl.x + vl.y);
        }
      }
      store(kr[x], row, k0, a);
    }
  }
}

// FP32 column weights 4 a0 omega_d v_d of dimension d into shared memory (zero padded),
// entries [lo, hi) of [0, npad); under the Gauss rule 4 a0 omega_q (Phi_d v_d) at the points.
__device__ inline void tc_weights(const StepParams& P, const KCompressed& kc, int d, float* w, int npad,
                                  int lo, int hi, int tid, int nthr) {
  const Dim& dd = P.d[d];
  const float s = static_cast<float>(4.0 * P.a0);
  if (hi > npad) hi = npad;
  if (P.quad) {
    for (int r = lo + tid; r < hi; r += nthr) {
      float v = 0.f;
      if (r < dd.nq) {
        float acc = 0.f;
        const int j0 = dd.phi0[r];
        for (int k = 0; k <= dd.b; ++k)
          if (j0 + k < dd.n) {
            const float2 ph = dd.phi[static_cast<size_t>(r) * kPhiW + k], vv = dd.v[j0 + k];
            acc = __fmaf_rn(ph.x + ph.y, vv.x + vv.y, acc);
          }
        v = static_cast<float>(dd.wq[r]) * acc;
      }
      w[r] = v;
    }
    return;
  }
  constexpr int kGroup = 8;   // loads of eight entries first, so that their latencies overlap
  for (int i0 = lo + tid; i0 < hi; i0 += kGroup * nthr) {
    float2 x[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      const int i = i0 + g * nthr;
      x[g] = i < dd.n ? dd.v[i] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      const int i = i0 + g * nthr;
      if (i < hi) w[i] = i < dd.n ? kc_omega(kc, i).x * (x[g].x + x[g].y) : 0.f;
    }
  }
}

// Cube form of the contraction (ctd_config.contraction_form).  With c_j the column weight of
// column j (the product of the other dimensions' tc_weights), the column operand's row j is
// scaled by cbrt(c_j) (the real cube root, sign kept), so that the tensor cores yield
// v_ij = cbrt(c_j) u_ij and the epilogue sums v^3 = c_j u_ij^3 with no weights.  The linear
// part sum_j c_j u_ij = sum_m a_m,i H_m (H_m the product of the Gram sums h_d,m = c_d . a_m,d)
// is subtracted exactly in the right-hand side.  The bound below selects the form per step
// in automatic mode: at |u| <= 0.6, |u^3| <= 0.36 |u|, so the cube sum cancels little against
// the linear part, and the split's rounding enters through 3 u^2 instead of |3 u^2 - 1|.
constexpr float kCubeMaxAmp = 0.6f;

// sum_m prod_d max_i |a_m,d(i)| over u^k's factors (at the nodes, or at the Gauss points),
// a bound of max |u^k| over the grid.  Every CTA computes it alike (exact maxima, then one
// thread's fixed-order sum), so all CTAs take the same decision.  s: dim * Mk floats of shared
// memory.
static __device__ __noinline__ float tc_amp_bound(const StepParams& P, int pb, int Mk, float* s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = warp; t < P.dim * Mk; t += nw) {
    const int d = t / Mk, m = t - d * Mk;
    const Dim& dd = P.d[d];
    const float2* src = (P.quad ? dd.Aq : dd.bank[pb]) + static_cast<size_t>(m) * dd.nq;
    float mx = 0.f;
    for (int i = lane; i < dd.nq; i += 32) {
      const float2 v = src[i];
      mx = fmaxf(mx, fabsf(v.x + v.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s[t] = mx;
  }
  __syncthreads();
  float B = 0.f;
  for (int m = 0; m < Mk; ++m) {
    float p = 1.f;
    for (int d = 0; d < P.dim; ++d) p *= s[d * Mk + m];
    B += p;
  }
  __syncthreads();
  return B;
}

// The cube form's column operand of direction x, written to `out` in the tile-image layout of
// tc_prepare: row j of the other dimension (2D), or row (j, l) = j n_last_pad + l of the middle
// and last dimensions (3D), times cbrt of its column weight.  The scale vectors are staged in
// shared memory s (ncols_pad floats in 2D; n_last_pad + nq_mid in 3D); the (row block, K step)
// pieces are spread over all warps of all CTAs.
static __device__ __noinline__ void tc_prepare_scaled(const StepParams& P, const KCompressed* kc, const TcDir& td,
                                                      __nv_bfloat16* out, int pb, int Mk, float* s) {
  const int KS = P.Kpad / 16, ksteps = (Mk + 15) / 16, nimg = tc_nimg(P.precision);
  if (ksteps == 0) return;
  const bool three = td.mid >= 0;
  const int nl = three ? td.n_last_pad : td.ncols_pad;
  const int nm = three ? P.d[td.mid].nq : 0;
  float* sl = s;
  float* sm = s + nl;
  tc_weights(P, kc[td.last], td.last, sl, nl, 0, nl, threadIdx.x, blockDim.x);
  if (three) tc_weights(P, kc[td.mid], td.mid, sm, nm, 0, nm, threadIdx.x, blockDim.x);
  __syncthreads();
  for (int i = threadIdx.x; i < nl + nm; i += blockDim.x) s[i] = cbrtf(s[i]);
  __syncthreads();
  auto src_of = [&](const Dim& dd) { return P.quad ? dd.Aq : dd.bank[pb]; };
  const Dim& dl = P.d[td.last];
  const float2* fl = src_of(dl);
  const float2* fm = three ? src_of(P.d[td.mid]) : nullptr;
  // one warp per (128-row block, K step); in 3D a block lies at one middle index j (n_last_pad
  // is a multiple of 128).  Lane: row rr = lane & 7 of each 8-row group, K half cm, and every
  // other group starting at gg; its eight K columns' middle factor is loaded once per block.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int rr = lane & 7, cm = (lane >> 3) & 1, gg = lane >> 4;
  const int nblk = td.ncols_pad / kTcM, work = nblk * ksteps;
  for (int wi = P.vrank * nw + warp; wi < work; wi += P.vgrid * nw) {
    const int blk = wi / ksteps, ks = wi - blk * ksteps;
    const int row0 = blk * kTcM;
    int j = 0, l0 = row0;
    if (three) {
      j = row0 / td.n_last_pad;
      l0 = row0 - j * td.n_last_pad;
    }
    const int k0 = ks * 16 + cm * 8;
    float fk[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      fk[e] = 0.f;
      if (k < Mk) {
        fk[e] = 1.f;
        if (three) {
          const float2 vm = fm[static_cast<size_t>(k) * nm + j];
          fk[e] = sm[j] * (vm.x + vm.y);
        }
      }
    }
    // every load of the block first (64 per lane in flight), then the products and stores: the
    // stores could alias the loads for the compiler, which would otherwise keep them in order
    float2 vl[8][8];
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int l = l0 + (gg + 2 * it) * 8 + rr;
#pragma unroll
      for (int e = 0; e < 8; ++e)
        vl[it][e] = (l < dl.nq && k0 + e < Mk) ? fl[static_cast<size_t>(k0 + e) * dl.nq + l] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int g = gg + 2 * it, l = l0 + g * 8 + rr;
      const float sc = l < dl.nq ? sl[l] : 0.f;
      float a[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) a[e] = sc * fk[e] * (vl[it][e].x + vl[it][e].y);
      // the BF16 terms of the split, as in tc_prepare
      const size_t o = tc_img_index(row0 + g * 8 + rr, k0, 0, KS, nimg);
      for (int h = 0; h < nimg; ++h) {
        __align__(16) __nv_bfloat16 t[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          t[e] = __float2bfloat16_rn(a[e]);
          a[e] -= __bfloat162float(t[e]);
        }
        *reinterpret_cast<uint4*>(out + o + static_cast<size_t>(h) * kTcImgElems) = *reinterpret_cast<const uint4*>(t);
      }
    }
  }
}

// Arena layout of the contraction phase (offsets from a 1024-byte aligned base)
struct TcLayout {
  size_t shared_off, a_off, b_off, wl_off, wm_off, total;
};
__host__ __device__ inline TcLayout tc_layout(int chunks, int stages, int wlast_n, int wmid_n) {
  TcLayout L;
  L.shared_off = 0;
  L.a_off = 1024;
  L.b_off = L.a_off + static_cast<size_t>(chunks) * kTcChunkBytes;
  L.wl_off = L.b_off + static_cast<size_t>(stages) * chunks * kTcChunkBytes;
  L.wm_off = L.wl_off + (static_cast<size_t>(wlast_n) * 4 + 127) / 128 * 128;
  L.total = L.wm_off + (static_cast<size_t>(wmid_n) * 4 + 127) / 128 * 128;
  return L;
}

// This CTA's share of the contraction for direction x.  Partial row sums go to
// rpart_tc[row * cmax + (cta - first owner of the row block)].  If dump != null the raw
// reconstructed values are written to dump[row * ncols_pad + col] instead (test probe).
// Returns false if a wait expired.
//
// Reduced integration domain (Section 3.3), 2D: with tile_max != null only the tiles whose
// stored max |u(u^2 - 1)| times on_scale (4 a0) exceeds on_tol are contracted; the others
// add nothing (their rows still get their partial sums written).  tile_max is indexed by
// the tile of direction 0 (row block of dimension 0, column block of dimension 1).
static __device__ __noinline__ bool tc_contract(const StepParams& P, const KCompressed* kc, const TcDir& td,
                                   const __nv_bfloat16* Pop, const __nv_bfloat16* Qop, int x, int Mk, int stages,
                                   unsigned char* base, uint32_t tmem_base, double* rpart_tc, float* dump,
                                   const unsigned* tile_max = nullptr, float on_scale = 0.f, float on_tol = 0.f,
                                   bool cube = false) {
  const int G = P.vgrid, cta = P.vrank;
  // Parameters the role loops use, in registers: P and td live in shared memory, and every
  // asm statement below (waits, MMAs, commits) is a memory clobber that would reload them.
  const int ntc = td.ntc, nrb = td.nrb, tmid = td.mid, cmax = td.cmax, n_last_pad = td.n_last_pad;
  const int ncols_pad = td.ncols_pad, nx = P.d[x].nq;
  InstState* const st = P.st;
  // Reduced domain: the 128-node block of every dimension that tile t lies in (in 3D a tile is
  // 128 rows of x by 128 nodes of the last dimension at one node of the middle one), blocks
  // numbered row-major over dimensions 0, 1 (, 2)
  const int nb1 = (P.d[1].n + kTcM - 1) / kTcM, nb2 = P.dim == 3 ? (P.d[2].n + kTcM - 1) / kTcM : 1;
  auto active = [=](int t) -> bool {
    if (!tile_max) return true;
    const int rb = t / ntc, cb = t - rb * ntc;
    int idx;
    if (tmid < 0) {
      idx = x == 0 ? t : cb * nrb + rb;
    } else {
      const int col0 = cb * kTcN, jm = col0 / n_last_pad;
      const int bm = jm / kTcM, bl = (col0 - jm * n_last_pad) / kTcN;
      auto blk = [&](int d) { return d == x ? rb : (d == tmid ? bm : bl); };
      idx = (blk(0) * nb1 + blk(1)) * nb2 + blk(2);
    }
    return __uint_as_float(tile_max[idx]) * on_scale > on_tol;
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nimg = tc_nimg(P.precision), npairs = tc_npairs(nimg);
  const int chunks = nimg * P.Kpad / kTcChunkElems;
  const int ksteps = (Mk + 15) / 16;
  // a block's images of the K steps that hold modes: one contiguous bulk copy
  const uint32_t load_bytes = static_cast<uint32_t>(nimg) * ksteps * kTcImgBytes;
  const size_t block_elems = static_cast<size_t>(P.Kpad / 16) * nimg * kTcImgElems;
  const int wl_n = tmid < 0 ? ncols_pad : n_last_pad;
  const int wm_n = tmid < 0 ? 0 : P.d[tmid].nq;
  const TcLayout Ly = tc_layout(chunks, stages, wl_n, wm_n);
  TcShared* sh = reinterpret_cast<TcShared*>(base + Ly.shared_off);
  unsigned char* As = base + Ly.a_off;
  unsigned char* Bs = base + Ly.b_off;
  float* wl = reinterpret_cast<float*>(base + Ly.wl_off);
  float* wm = reinterpret_cast<float*>(base + Ly.wm_off);
  const long long T = static_cast<long long>(nrb) * ntc;
  const int t0 = tile_lo(T, G, cta), t1 = tile_lo(T, G, cta + 1);
  const unsigned long long lim = P.wait_ns;
  const uint32_t stage_bytes = static_cast<uint32_t>(chunks) * kTcChunkBytes;
  // role timing (SM cycles) on the traced CTA: the last one, whose tile share is a full one
  unsigned long long* const tr = (P.trace && cta == G - 1) ? P.trace : nullptr;
  long long t_wait = 0, t_wait2 = 0, t_work = 0;

  if (threadIdx.x == 0) {
    mbar_init(&sh->a_full, 1);
    mbar_init(&sh->a_empty, 1);
    for (int s = 0; s < stages; ++s) { mbar_init(&sh->b_full[s], 1); mbar_init(&sh->b_empty[s], 1); }
    for (int a = 0; a < kTcAcc; ++a) { mbar_init(&sh->acc_full[a], 1); mbar_init(&sh->acc_empty[a], 128); }
    sh->abort = 0;
    fence_barrier_init();
  }
  // The arena held generic-proxy data of earlier phases (Gram staging, solver vectors) where
  // the bulk copies and the MMAs now write and read through the async proxy: every thread
  // orders its earlier shared-memory accesses before them.
  fence_proxy_async();
  __syncthreads();
  if (Mk == 0 || ksteps == 0) {
    // u^k = 0: w(0) = 0, every partial is zero
    if (!dump) {
      for (long long t = t0; t < t1; ++t) {
        const int rb = static_cast<int>(t / ntc);
        if (t != t0 && t / ntc == (t - 1) / ntc) continue;
        const int j = cta - tile_owner(T, G, static_cast<long long>(rb) * ntc);
        for (int r = threadIdx.x; r < kTcM; r += blockDim.x) {
          const int row = rb * kTcM + r;
          if (row < nx) rpart_tc[static_cast<size_t>(row) * cmax + j] = 0.0;
        }
      }
    }
    __syncthreads();
    return true;
  }
  volatile int* abort_flag = &sh->abort;
  bool ok = true;

  // Tiles go through the pipeline in groups: two consecutive column blocks of one row block
  // when no tile is skipped and a stage holds both tiles' images, else one tile.  A group
  // takes one ring stage (its tiles' images side by side) and one of two accumulator pairs
  // (TMEM columns [256 p, 256 p + 256)), so each barrier wait and commit covers a group.
  const bool pairs = !tile_max && 2 * load_bytes <= stage_bytes;
  auto group_size = [=](int t, int cb) -> int { return (pairs && t + 1 < t1 && cb + 1 < ntc) ? 2 : 1; };

  // The producer and MMA warps walk their loops with all lanes (waits by the whole warp, so
  // that it stays converged); lane 0 issues the copies, the MMAs and the commits.
  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) fence_proxy_async_global();     // operands were written through the generic proxy
    int cur_rb = -1, a_loads = 0;
    int rb = t0 / ntc, cb = t0 - rb * ntc;   // row and column block of tile t, kept incrementally
    int s = 0, round = 0, gi = 0;            // ring stage of the next group, its round, group count
    for (int t = t0, g = 1; t < t1 && ok; t += g, cb += g, rb += (cb >= ntc), cb -= (cb >= ntc) ? ntc : 0) {
      g = 1;
      if (!active(t)) continue;
      g = group_size(t, cb);
      if (rb != cur_rb) {
        if (a_loads > 0 && !warp_wait(&sh->a_empty, (a_loads - 1) & 1, lim, st, abort_flag, 21)) { ok = false; break; }
        if (lane == 0) {
          mbar_expect_tx(&sh->a_full, load_bytes);
          bulk_load(As, Pop + static_cast<size_t>(rb) * block_elems, load_bytes, &sh->a_full);
        }
        __syncwarp();
        ++a_loads;
        cur_rb = rb;
      }
      const long long c0 = tr ? clock64() : 0;
      if (gi >= stages && !warp_wait(&sh->b_empty[s], (round - 1) & 1, lim, st, abort_flag, 22)) { ok = false; break; }
      if (tr) t_wait += clock64() - c0;
      if (lane == 0) {
        mbar_expect_tx(&sh->b_full[s], g * load_bytes);
        for (int j = 0; j < g; ++j)
          bulk_load(Bs + static_cast<size_t>(s) * stage_bytes + j * load_bytes,
                    Qop + static_cast<size_t>(cb + j) * block_elems, load_bytes, &sh->b_full[s]);
      }
      __syncwarp();
      ++gi;
      if (++s == stages) { s = 0; ++round; }
    }
    if (!ok && lane == 0) sh->abort = 1;
    if (tr && lane == 0) atomicAdd(tr + kTrTcProdWait, static_cast<unsigned long long>(t_wait));
  } else if (warp == 1) {
    // ---------------- MMA issuer
    const uint32_t idesc = umma_idesc_bf16();
    const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
    int cur_rb = -1, a_uses = 0, n_g = 0;
    int rb = t0 / ntc, cb = t0 - rb * ntc;
    int s = 0, round = 0, gi = 0;
    for (int t = t0, g = 1; t < t1 && ok; t += g, cb += g, rb += (cb >= ntc), cb -= (cb >= ntc) ? ntc : 0) {
      g = 1;
      if (!active(t)) continue;
      g = group_size(t, cb);
      if (rb != cur_rb) {
        if (!warp_wait(&sh->a_full, a_uses & 1, lim, st, abort_flag, 23)) { ok = false; break; }
        ++a_uses;
        cur_rb = rb;
      }
      const long long c0 = tr ? clock64() : 0;
      if (!warp_wait(&sh->b_full[s], round & 1, lim, st, abort_flag, 24)) { ok = false; break; }
      const long long c1 = tr ? clock64() : 0;
      const int ps = gi & 1;   // accumulator pair
      if (gi >= 2 && !warp_wait(&sh->acc_empty[ps], ((gi >> 1) - 1) & 1, lim, st, abort_flag, 25)) {
        ok = false;
        break;
      }
      const long long c2 = tr ? clock64() : 0;
      if (tr) { t_wait += c1 - c0; t_wait2 += c2 - c1; }
      tc_fence_after();
      // is this the row block's last contracted group (then its A block is released)?
      bool last_in_rb;
      if (!tile_max) {
        last_in_rb = t + g == t1 || cb + g == ntc;
      } else {
        int tn = t + 1;   // next tile that is contracted
        while (tn < t1 && !active(tn)) ++tn;
        last_in_rb = tn == t1 || tn / ntc != rb;
      }
      if (lane == 0) {
        for (int j = 0; j < g; ++j) {
          const uint32_t d = tmem_base + static_cast<uint32_t>((2 * ps + j) * kTcN);
          const uint32_t bs = b_base + static_cast<uint32_t>(s) * stage_bytes + j * load_bytes;
          for (int k = 0; k < ksteps; ++k) {
            const uint32_t off = static_cast<uint32_t>(k * nimg) * kTcImgBytes;
            for (int p = 0; p < npairs; ++p) {
              const uint64_t ad = umma_desc_img(a_base + off + tc_pair_a(p) * kTcImgBytes);
              const uint64_t bd = umma_desc_img(bs + off + tc_pair_b(p) * kTcImgBytes);
              tc_mma(d, ad, bd, idesc, (k > 0 || p > 0) ? 1u : 0u);
            }
          }
        }
        tc_commit(&sh->b_empty[s]);
        tc_commit(&sh->acc_full[ps]);
        if (last_in_rb) tc_commit(&sh->a_empty);
      }
      __syncwarp();
      if (tr) t_work += clock64() - c2;
      ++gi;
      n_g = gi;
      if (++s == stages) { s = 0; ++round; }
    }
    if (tr && lane == 0) {
      atomicAdd(tr + kTrTcMmaWaitB, static_cast<unsigned long long>(t_wait));
      atomicAdd(tr + kTrTcMmaWaitAcc, static_cast<unsigned long long>(t_wait2));
      atomicAdd(tr + kTrTcMmaIssue, static_cast<unsigned long long>(t_work));
      atomicAdd(tr + kTrTcTiles, static_cast<unsigned long long>(t1 - t0));
    }
    if (!ok) {
      if (lane == 0) sh->abort = 1;
    } else if (n_g > 0) {
      // quiesce: the last commits have landed before the barriers are re-initialised
      for (int q = 0; q < stages && q < n_g; ++q) {
        const int last_g = q + ((n_g - 1 - q) / stages) * stages;
        if (!warp_wait(&sh->b_empty[q], (last_g / stages) & 1, lim, st, abort_flag, 26)) { ok = false; break; }
      }
      if (ok && !warp_wait(&sh->a_empty, (a_uses - 1) & 1, lim, st, abort_flag, 27)) ok = false;
      if (!ok && lane == 0) sh->abort = 1;
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: one TMEM lane (tile row) per thread
    const int r = (warp - 4) * 32 + lane;
    // column weights of the fixed factors (in 2D only those of this CTA's column blocks),
    // formed by the epilogue's 128 threads while the first copies and MMAs are in flight
    if (cube) {
    } else if (tmid >= 0) {
      tc_weights(P, kc[td.last], td.last, wl, wl_n, 0, wl_n, r, 128);
      tc_weights(P, kc[tmid], tmid, wm, wm_n, 0, wm_n, r, 128);
    } else if (t1 - t0 >= ntc) {
      tc_weights(P, kc[td.last], td.last, wl, wl_n, 0, wl_n, r, 128);
    } else if (t1 > t0) {
      const int cb_lo = t0 % ntc, cb_hi = (t1 - 1) % ntc;
      if (cb_lo <= cb_hi) {
        tc_weights(P, kc[td.last], td.last, wl, wl_n, cb_lo * kTcN, (cb_hi + 1) * kTcN, r, 128);
      } else {   // the range wraps into the next row block
        tc_weights(P, kc[td.last], td.last, wl, wl_n, 0, (cb_hi + 1) * kTcN, r, 128);
        tc_weights(P, kc[td.last], td.last, wl, wl_n, cb_lo * kTcN, wl_n, r, 128);
      }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");   // the epilogue warps only
    const uint32_t lane_base = tmem_base + (static_cast<uint32_t>((warp & 3) * 32) << 16);
    // FP32 within a tile, double-float (two FP32 words, exact products) across the tiles of a
    // row block: hundreds of tiles whose sums cancel would lose the FP32 sum's digits
    dfloat acc = {0.f, 0.f};
    int cur_rb = -1;
    auto flush = [&](int rbf) {
      const int row = rbf * kTcM + r;
      if (!dump && row < nx) {
        const int j = cta - tile_owner(T, G, static_cast<long long>(rbf) * ntc);
        rpart_tc[static_cast<size_t>(row) * cmax + j] = static_cast<double>(acc.hi) + static_cast<double>(acc.lo);
      }
    };
    int rb = t0 / ntc, cb = t0 - rb * ntc;
    int gi = 0;
    for (int t = t0, g = 1; t < t1; t += g, cb += g, rb += (cb >= ntc), cb -= (cb >= ntc) ? ntc : 0) {
      g = 1;
      if (rb != cur_rb) {
        if (cur_rb >= 0) flush(cur_rb);
        acc = {0.f, 0.f};
        cur_rb = rb;
      }
      if (!active(t)) continue;
      g = group_size(t, cb);
      const int ps = gi & 1;
      // each lane leaves its wait on its own; the TMEM loads below are warp-collective
      // (.sync.aligned), so the warp reconverges (and agrees on the outcome) first
      const long long c0 = tr ? clock64() : 0;
      if (!warp_wait(&sh->acc_full[ps], (gi >> 1) & 1, lim, st, abort_flag, 28)) { ok = false; break; }
      const long long c1 = tr ? clock64() : 0;
      ++gi;
      tc_fence_after();
      for (int j = 0; j < g && cube; ++j) {
        // cube form: v^3 = c_j u^3, two columns per FP32x2 instruction, four interleaved sums
        float2 a01 = make_float2(0.f, 0.f), a23 = a01, b01 = a01, b23 = a01;
        const uint32_t acol = static_cast<uint32_t>((2 * ps + j) * kTcN);
#pragma unroll
        for (int q = 0; q < kTcN / 32; ++q) {
          float v[32];
          tmem_ld32(lane_base + acol + static_cast<uint32_t>(q * 32), v);
#pragma unroll
          for (int c = 0; c < 32; c += 8) {
            const float2 u01 = make_float2(v[c], v[c + 1]), u23 = make_float2(v[c + 2], v[c + 3]);
            const float2 u45 = make_float2(v[c + 4], v[c + 5]), u67 = make_float2(v[c + 6], v[c + 7]);
            a01 = __ffma2_rn(__fmul2_rn(u01, u01), u01, a01);
            a23 = __ffma2_rn(__fmul2_rn(u23, u23), u23, a23);
            b01 = __ffma2_rn(__fmul2_rn(u45, u45), u45, b01);
            b23 = __ffma2_rn(__fmul2_rn(u67, u67), u67, b23);
          }
        }
        const float at = ((a01.x + a01.y) + (a23.x + a23.y)) + ((b01.x + b01.y) + (b23.x + b23.y));
        acc = df_add(acc, dfloat{at, 0.f});
      }
      for (int j = 0; j < g && !cube; ++j) {
        const int col0 = (cb + j) * kTcN;
        const float* wt;
        float wscale = 1.f;
        if (tmid < 0) {
          wt = wl + col0;
        } else {
          const int jm = col0 / n_last_pad;
          wt = wl + (col0 - jm * n_last_pad);
          wscale = wm[jm];
        }
        // w(u)/(4 a0) = u (u^2 - 1) and the weighted row sum, two columns per FP32x2
        // instruction; four interleaved sums (columns 0, 1, 2, 3 mod 4)
        float2 a01 = make_float2(0.f, 0.f), a23 = a01, b01 = a01, b23 = a01;
        const float2 m1 = make_float2(-1.f, -1.f);
        const uint32_t acol = static_cast<uint32_t>((2 * ps + j) * kTcN);
#pragma unroll
        for (int q = 0; q < kTcN / 32; ++q) {
          float v[32];
          tmem_ld32(lane_base + acol + static_cast<uint32_t>(q * 32), v);
          if (dump) {
            const int row = rb * kTcM + r;
            for (int c = 0; c < 32; ++c) dump[static_cast<size_t>(row) * ncols_pad + col0 + q * 32 + c] = v[c];
          }
          const float4* w4 = reinterpret_cast<const float4*>(wt + q * 32);
#pragma unroll
          for (int c = 0; c < 8; c += 2) {
            const float4 wa = w4[c], wb = w4[c + 1];
            const float2 u01 = make_float2(v[4 * c], v[4 * c + 1]), u23 = make_float2(v[4 * c + 2], v[4 * c + 3]);
            const float2 u45 = make_float2(v[4 * c + 4], v[4 * c + 5]), u67 = make_float2(v[4 * c + 6], v[4 * c + 7]);
            // w u (u^2 - 1): the weight product and u^2 - 1 are independent, so each column pair
            // has a chain of two dependent operations before its accumulator
            a01 = __ffma2_rn(__fmul2_rn(u01, make_float2(wa.x, wa.y)), __ffma2_rn(u01, u01, m1), a01);
            a23 = __ffma2_rn(__fmul2_rn(u23, make_float2(wa.z, wa.w)), __ffma2_rn(u23, u23, m1), a23);
            b01 = __ffma2_rn(__fmul2_rn(u45, make_float2(wb.x, wb.y)), __ffma2_rn(u45, u45, m1), b01);
            b23 = __ffma2_rn(__fmul2_rn(u67, make_float2(wb.z, wb.w)), __ffma2_rn(u67, u67, m1), b23);
          }
        }
        const float at = ((a01.x + a01.y) + (a23.x + a23.y)) + ((b01.x + b01.y) + (b23.x + b23.y));
        const float pr = wscale * at;
        acc = df_add(acc, dfloat{pr, __fmaf_rn(wscale, at, -pr)});
      }
      tc_fence_before();
      mbar_arrive(&sh->acc_empty[ps]);
      if (tr) { t_wait += c1 - c0; t_work += clock64() - c1; }
    }
    if (ok && cur_rb >= 0) flush(cur_rb);
    if (!ok) sh->abort = 1;
    if (tr && warp == 4 && lane == 0) {
      atomicAdd(tr + kTrTcEpiWait, static_cast<unsigned long long>(t_wait));
      atomicAdd(tr + kTrTcEpiWork, static_cast<unsigned long long>(t_work));
    }
  }
  __syncthreads();
  return !(*abort_flag);
}

}  // namespace ctd

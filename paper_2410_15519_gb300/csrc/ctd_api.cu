// C ABI of the CTD solver (declared in include/ctd.h): workspace layout, handle, launches.
#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "ctd.h"
#include "cfem_host.h"
#include "ctd_actd.h"
#include "ctd_kernels.h"

using ctd::Dim;
using ctd::Extra;
using ctd::InstState;
using ctd::StepParams;
using ctd::StepStatsDev;

namespace {

constexpr int kGridMax = 512;        // largest persistent grid the workspace is sized for
constexpr int kStatsCap = 256;       // step records kept on the device between reads

// Bump allocator over the caller's workspace (256-byte aligned pieces).  With base == null
// it only measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~static_cast<size_t>(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * count;
    return p;
  }
};

struct Plan {
  int D, n[3], nq[3], quad, b[3], n_pad[3], Mcap, Kpad, sep_q, grid, rchunks[3];
  long long N;
  size_t rpart_len, rpart_tc_len;
  ctd::TcDir dirs[3];
};

// Tensor-core geometry of direction x for a grid of G CTAs.
ctd::TcDir tc_dir(const Plan& p, int x, int G) {
  ctd::TcDir t{};
  t.nrb = p.n_pad[x] / ctd::kTcM;
  if (p.D == 2) {
    t.mid = -1;
    t.last = 1 - x;
    t.ncols_pad = p.n_pad[t.last];
    t.n_last_pad = p.n_pad[t.last];
  } else {
    t.mid = x == 0 ? 1 : 0;
    t.last = x == 2 ? 1 : 2;
    t.n_last_pad = p.n_pad[t.last];
    t.ncols_pad = p.nq[t.mid] * t.n_last_pad;
  }
  t.ntc = t.ncols_pad / ctd::kTcN;
  const long long T = static_cast<long long>(t.nrb) * t.ntc;
  int cmax = 1;
  for (int rb = 0; rb < t.nrb; ++rb) {
    const int c0 = ctd::tile_owner(T, G, static_cast<long long>(rb) * t.ntc);
    const int c1 = ctd::tile_owner(T, G, static_cast<long long>(rb) * t.ntc + t.ntc - 1);
    cmax = std::max(cmax, c1 - c0 + 1);
  }
  t.cmax = cmax;
  return t;
}

int half_bandwidth(int s) { return 2 * s + 1; }

// Chunks of the FP64 contraction for direction x over a grid of nd[] points per dimension
int chunks_for(int D, const int* nd, int x, int grid) {
  const int nc = nd[x];
  const long long tw = static_cast<long long>(grid) * ctd::kWarps;
  long long C;
  if (x == D - 1) {
    long long rows = 1;
    for (int d = 0; d < D; ++d)
      if (d != x) rows *= nd[d];
    const long long cblocks = (nc + 31) / 32;
    C = std::min<long long>(rows, std::max<long long>(1, (4 * tw + cblocks - 1) / cblocks));
  } else {
    const int extent = (D == 2) ? nd[1] : (x == 0 ? nd[1] : nd[0]);
    C = std::min<long long>(extent, std::max<long long>(1, (4 * tw + nc - 1) / nc));
  }
  return static_cast<int>(C);
}

Plan make_plan(const ctd_config& c, int grid) {
  Plan p{};
  p.D = c.dim;
  p.N = 1;
  p.quad = c.quad_rule == CTD_QUAD_GAUSS ? 1 : 0;
  for (int d = 0; d < c.dim; ++d) {
    p.n[d] = c.n[d];
    // grid of the nonlinear term: the nodes, or q Gauss points per element
    p.nq[d] = p.quad ? c.quad_q * (c.n[d] - 1) : c.n[d];
    p.b[d] = half_bandwidth(c.s);
    p.n_pad[d] = (p.nq[d] + ctd::kTileRows - 1) / ctd::kTileRows * ctd::kTileRows;
    p.N *= p.nq[d];
  }
  p.Mcap = c.M_max;
  p.Kpad = (c.M_max + 63) / 64 * 64;
  p.sep_q = c.nonlinear_form == CTD_NONLINEAR_SEPARATED ? ctd::sep_terms(c.M_max) : 0;
  p.grid = grid;
  p.rpart_len = 0;
  p.rpart_tc_len = 0;
  for (int x = 0; x < c.dim; ++x) {
    p.rchunks[x] = chunks_for(c.dim, p.nq, x, grid);
    p.rpart_len = std::max(p.rpart_len, static_cast<size_t>(p.nq[x]) * p.rchunks[x]);
  }
  for (int x = 0; x < c.dim; ++x) {
    p.dirs[x] = tc_dir(p, x, grid);
    p.rpart_tc_len = std::max(p.rpart_tc_len, static_cast<size_t>(p.nq[x]) * p.dirs[x].cmax);
  }
  return p;
}

// Lay out every workspace piece; fills P and X pointers when base != null.
size_t carve(const ctd_config& c, const Plan& pl, void* base, StepParams* P, Extra* X,
             float2** kc_store, float2** mc_store, double** energy_part, double** energy_gram,
             StepStatsDev** stats, ctd::ActdState* actd) {
  Carver cv(base);
  StepParams p{};
  Extra x{};
  const int D = c.dim;
  // sizing uses the largest grid so one workspace fits any grid choice
  const int Gs = kGridMax;
  for (int d = 0; d < D; ++d) {
    const int n = pl.n[d], w = 2 * pl.b[d] + 1;
    Dim& dd = p.d[d];
    dd.n = n;
    dd.b = pl.b[d];
    dd.n_pad = pl.n_pad[d];
    dd.omega = cv.take<double>(n);
    dd.kband = cv.take<double>(static_cast<size_t>(n) * w);
    dd.bank[0] = cv.take<float2>(static_cast<size_t>(pl.Mcap) * n);
    dd.bank[1] = cv.take<float2>(static_cast<size_t>(pl.Mcap) * n);
    dd.KB = cv.take<float2>(static_cast<size_t>(pl.Mcap) * n);
    dd.v = cv.take<float2>(n);
    dd.vold = cv.take<float2>(n);
    dd.op = (c.precision != CTD_PREC_FP64)
                ? cv.take<__nv_bfloat16>(static_cast<size_t>(pl.n_pad[d]) * ctd::tc_nimg(c.precision) * pl.Kpad)
                : nullptr;
    kc_store[d] = cv.take<float2>(static_cast<size_t>(n + 1) * w);
    x.Af[d] = cv.take<double>(static_cast<size_t>(pl.Mcap) * n);
    dd.nq = pl.nq[d];
    if (pl.quad) {
      const int nq = pl.nq[d];
      dd.wq = cv.take<double>(nq);
      dd.phi = cv.take<float2>(static_cast<size_t>(nq) * ctd::kPhiW);
      dd.phi0 = cv.take<int>(nq);
      dd.mband = cv.take<double>(static_cast<size_t>(n) * w);
      dd.MA = cv.take<float2>(static_cast<size_t>(pl.Mcap) * n);
      dd.MB = cv.take<float2>(static_cast<size_t>(pl.Mcap) * n);
      dd.Aq = cv.take<float2>(static_cast<size_t>(pl.Mcap) * nq);
      mc_store[d] = cv.take<float2>(static_cast<size_t>(n + 1) * w);
    } else {
      mc_store[d] = nullptr;
    }
  }
  int nmax = 0;
  for (int d = 0; d < D; ++d) nmax = std::max(nmax, pl.n[d]);
  const int spd = ctd::slots_per_dim(pl.Mcap, pl.sep_q);
  const int nslots = std::max((D - 1) * spd, D * 6);
  p.gram = cv.take<float2>(static_cast<size_t>(nslots) * Gs);
  p.rpart = cv.take<double>(std::max(pl.rpart_len, static_cast<size_t>(nmax)));   // also the probe's linear part
  x.rpart_tc = cv.take<double>(std::max<size_t>(1, pl.rpart_tc_len));
  for (int k = 0; k < 3; ++k) x.kr[k] = nullptr;
  // column operands per direction: the 3D Khatri-Rao products, and the cube form's scaled
  // operand (2D and 3D)
  if (c.precision != CTD_PREC_FP64)
    for (int k = 0; k < D; ++k)
      x.kr[k] = cv.take<__nv_bfloat16>(static_cast<size_t>(pl.dirs[k].ncols_pad) * ctd::tc_nimg(c.precision) *
                                       pl.Kpad);
  for (int k = 0; k < D; ++k) x.dirs[k] = pl.dirs[k];
  p.Q = cv.take<float2>(ctd::kMaxN);
  size_t crf = 0;
  for (int d = 0; d < D; ++d)
    crf = std::max(crf, std::max(ctd::cr_floats(pl.n[d], pl.b[d]), ctd::l0_global_floats(pl.n[d], pl.b[d])));
  p.solver = cv.take<float>(crf);
  p.xsol_g = cv.take<float2>(ctd::kMaxN);
  p.W = (c.precision == CTD_PREC_FP64) ? cv.take<double>(static_cast<size_t>(pl.N)) : nullptr;
  p.U = nullptr;
  if (c.actd_Mc > 0) {
    // adaptive CTD: the full-grid field, a full-grid scratch, eigenpairs, eigensolver scratch
    ctd::ActdState a;
    p.U = cv.take<double>(static_cast<size_t>(pl.N));
    a.Y = cv.take<double>(static_cast<size_t>(pl.N));
    int nm = 0;
    for (int d = 0; d < D; ++d) {
      a.V[d] = cv.take<double>(static_cast<size_t>(pl.n[d]) * pl.n[d]);
      a.lam[d] = cv.take<double>(pl.n[d]);
      nm = std::max(nm, pl.n[d]);
    }
    a.work_len = ctd::actd_work_doubles(nm);
    a.work = cv.take<double>(a.work_len);
    a.info = cv.take<int>(64);
    if (actd) *actd = a;
  }
  p.barrier = cv.take<unsigned>(64);
  size_t nblocks = 1;   // reduced domain: 128-node blocks per dimension
  for (int d = 0; d < D; ++d) nblocks *= static_cast<size_t>(pl.n_pad[d] / ctd::kTcM);
  p.tile_max = cv.take<unsigned>(nblocks);
  p.trace = cv.take<unsigned long long>(ctd::kTrSlots);
  p.st = cv.take<InstState>(1);
  x.maxpart = cv.take<double>(static_cast<size_t>(ctd::kMaxDim) * Gs);
  x.xprev = cv.take<float2>(static_cast<size_t>(ctd::kMaxDim) * ctd::kMaxN);
  x.ctrl = cv.take<int>(64);
  *stats = cv.take<StepStatsDev>(kStatsCap);
  *energy_part = cv.take<double>(1024);
  *energy_gram = cv.take<double>(static_cast<size_t>(D) * 2 * pl.Mcap * pl.Mcap);
  if (P) *P = p;
  if (X) *X = x;
  return cv.off + 256;
}

const char* status_text(int s) {
  switch (s) {
    case CTD_OK: return "ok";
    case CTD_STATUS_CAPPED: return "a step reached the mode cap M_max";
    case CTD_STATUS_ALS_NOT_CONVERGED: return "a mode ended its sweeps without meeting tol_als (I_max or stall rule)";
    case CTD_ERR_ARG: return "invalid argument";
    case CTD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case CTD_ERR_CUDA: return "CUDA runtime error";
    case CTD_ERR_NONFINITE: return "non-finite value or failed factorisation";
    case CTD_ERR_TIMEOUT: return "a grid-wide wait exceeded its limit";
    case CTD_ERR_STATE: return "call out of order";
    case CTD_ERR_UNSUPPORTED: return "not supported by this build";
    default: return "unknown status";
  }
}

ctd_status validate(const ctd_config* c) {
  if (!c) return CTD_ERR_ARG;
  if (c->dim != 2 && c->dim != 3) return CTD_ERR_ARG;
  for (int d = 0; d < c->dim; ++d) {
    if (c->n[d] < 4 || c->n[d] > ctd::kMaxN) return CTD_ERR_ARG;
    if (!(c->length[d] > 0.0) || !std::isfinite(c->length[d])) return CTD_ERR_ARG;
  }
  if (c->s < 1 || c->s > 3 || c->p < 0 || c->p > c->s) return CTD_ERR_ARG;
  if (!(c->a > 0.0) || !(c->L > 0.0) || !(c->kappa > 0.0) || !(c->a0 >= 0.0) || !(c->alpha >= 0.0))
    return CTD_ERR_ARG;
  if (!(c->dt > 0.0) || !std::isfinite(c->dt)) return CTD_ERR_ARG;
  if (c->M_max < 1 || c->M_max > ctd::kMaxModes || c->I_max < 1) return CTD_ERR_ARG;
  if (!(c->tol_als >= 0.0) || !(c->tol_enrich >= 0.0)) return CTD_ERR_ARG;
  if (!(c->als_stall_tol >= 0.0) || !std::isfinite(c->als_stall_tol)) return CTD_ERR_ARG;
  if (c->fixed_als_iters < 0 || c->fixed_modes < 0 || c->fixed_modes > c->M_max) return CTD_ERR_ARG;
  if (c->precision != CTD_PREC_FP64 && c->precision != CTD_PREC_SPLIT_BF16 && c->precision != CTD_PREC_BF16 &&
      c->precision != CTD_PREC_SPLIT3_BF16)
    return CTD_ERR_ARG;
  if (c->grid_ctas > kGridMax) return CTD_ERR_ARG;
  if (!(c->reduced_tol >= 0.0) || !std::isfinite(c->reduced_tol)) return CTD_ERR_ARG;
  if (c->nonlinear_form != CTD_NONLINEAR_GRID && c->nonlinear_form != CTD_NONLINEAR_SEPARATED) return CTD_ERR_ARG;
  if (c->nonlinear_form == CTD_NONLINEAR_SEPARATED && (c->reduced_tol > 0.0 || c->M_max > ctd::kMaxSepModes))
    return CTD_ERR_ARG;
  if (c->quad_rule != CTD_QUAD_NODAL && c->quad_rule != CTD_QUAD_GAUSS) return CTD_ERR_ARG;
  if (c->actd_Mc < 0) return CTD_ERR_ARG;
  if (c->contraction_form < CTD_CONTRACT_AUTO || c->contraction_form > CTD_CONTRACT_CUBE) return CTD_ERR_ARG;
  if (c->actd_Mc > 0 && (c->precision != CTD_PREC_FP64 || c->quad_rule != CTD_QUAD_NODAL ||
                         c->nonlinear_form != CTD_NONLINEAR_GRID || c->reduced_tol > 0.0))
    return CTD_ERR_UNSUPPORTED;
  if (c->quad_rule == CTD_QUAD_GAUSS) {
    if (c->quad_q < 1 || c->quad_q > ctd::kMaxGaussPoints) return CTD_ERR_ARG;
    if (c->nonlinear_form != CTD_NONLINEAR_GRID || c->reduced_tol > 0.0) return CTD_ERR_UNSUPPORTED;
    // the FP64 contraction keeps the other dimensions' weights at their points in shared memory
    for (int x = 0; x < c->dim; ++x) {
      long long tot = 0;
      for (int d = 0; d < c->dim; ++d)
        if (d != x) tot += (static_cast<long long>(c->quad_q) * (c->n[d] - 1) + 1) & ~1LL;
      if (tot > static_cast<long long>(ctd::kMaxDim) * ctd::kMaxN) return CTD_ERR_UNSUPPORTED;
    }
  }
  return CTD_OK;
}

// Compressed band (double-float): rows [0, lead) and [n - tail, n) explicit, the interior
// rows [2s+1, n-2-2s] equal to one stencil when the mesh makes them identical (else every row
// explicit).  Layout: (lead + tail) rows, then the stencil.
std::vector<float2> compress_band(const std::vector<double>& band, int n, int s, int w, int* lead_out, int* tail_out) {
  int lead = 2 * s + 1, tail = 2 * s + 1;
  bool uniform = n > lead + tail;
  if (uniform) {
    const double* ref = &band[static_cast<size_t>(lead) * w];
    for (int i = lead; i < n - tail && uniform; ++i)
      for (int k = 0; k < w; ++k)
        if (band[static_cast<size_t>(i) * w + k] != ref[k]) { uniform = false; break; }
  }
  if (!uniform) { lead = n; tail = 0; }
  auto to_df = [](double v) {
    const float hi = static_cast<float>(v);
    return make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
  };
  std::vector<float2> kc(static_cast<size_t>(lead + tail + 1) * w);
  for (int i = 0; i < lead; ++i)
    for (int k = 0; k < w; ++k) kc[static_cast<size_t>(i) * w + k] = to_df(band[static_cast<size_t>(i) * w + k]);
  for (int t = 0; t < tail; ++t)
    for (int k = 0; k < w; ++k)
      kc[static_cast<size_t>(lead + t) * w + k] = to_df(band[static_cast<size_t>(n - tail + t) * w + k]);
  const int srow = uniform ? lead : 0;
  for (int k = 0; k < w; ++k) kc[static_cast<size_t>(lead + tail) * w + k] = to_df(band[static_cast<size_t>(srow) * w + k]);
  *lead_out = lead;
  *tail_out = tail;
  return kc;
}

}  // namespace

struct ctd_ctx {
  ctd_config cfg;
  cudaStream_t stream;
  int device;
  int grid;
  Plan plan;
  StepParams P;
  Extra X;
  float2* kc_store[3];
  float2* mc_store[3];
  std::vector<double> gphi[3];   // Gauss rule: shape function values at the points [nq][2s+2]
  std::vector<int> gcol0[3];     // and their first nodes
  std::vector<double> gwq[3];    // and the weights of the points
  ctd::ActdState actd;           // adaptive CTD: library handles, eigenpairs, scratch
  double* energy_part;
  double* energy_gram;
  StepStatsDev* stats_dev;
  unsigned long long* trace_dev;
  double mu_max[3];
  std::vector<double> omega[3], kband[3];
  bool has_modes;
  std::string err;
};

// message of the last ctd_create that failed after its checks (ctd_last_error(NULL)), per thread
static thread_local std::string g_create_err;

static ctd_status fail(ctd_ctx* h, ctd_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}
static ctd_status cuda_fail(ctd_ctx* h, cudaError_t e, const char* where) {
  return fail(h, CTD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CTD_CUDA(h, call)                                    \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

// Dump array of ctd_probe_reconstruct_noalloc: a file-scope device array (one instance per
// device, created with the module), for callers that cannot allocate device memory.  Its
// address is looked up once per device, with that device current, and cached.
static __device__ __align__(256) unsigned char g_static_dump[CTD_RECONSTRUCT_STATIC_BYTES];
namespace {
constexpr int kStaticDumpDevices = 64;
std::mutex g_static_dump_mu;
void* g_static_dump_ptr[kStaticDumpDevices] = {};
}  // namespace
static cudaError_t static_dump_address(int device, void** ptr) {
  if (device < 0 || device >= kStaticDumpDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_dump_mu);
  if (!g_static_dump_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_dump);
    if (e != cudaSuccess) return e;
    g_static_dump_ptr[device] = p;
  }
  *ptr = g_static_dump_ptr[device];
  return cudaSuccess;
}

static ctd_status status_from_bits(int bits) {
  if (bits & ctd::kErrTimeout) return CTD_ERR_TIMEOUT;
  if (bits & (ctd::kErrNonfinite | ctd::kErrSolve)) return CTD_ERR_NONFINITE;
  return CTD_OK;
}

extern "C" {

const char* ctd_status_string(int status) { return status_text(status); }

const char* ctd_last_error(ctd_handle h) {
  if (!h) return g_create_err.empty() ? "no handle" : g_create_err.c_str();
  return h->err.c_str();
}

ctd_status ctd_workspace_size(const ctd_config* cfg, size_t* bytes) {
  ctd_status v = validate(cfg);
  if (v != CTD_OK) return v;
  if (!bytes) return CTD_ERR_ARG;
  float2* kc[3];
  float2* mc[3];
  double *ep, *eg;
  StepStatsDev* sd;
  size_t best = 0;
  // every grid size 1..kGridMax fits (rpart_tc depends on the split of tiles over CTAs)
  for (int g : {1, 2, 4, 8, 16, 32, 64, 128, 132, 144, 148, 152, 160, 256, kGridMax}) {
    const Plan pl = make_plan(*cfg, g);
    best = std::max(best, carve(*cfg, pl, nullptr, nullptr, nullptr, kc, mc, &ep, &eg, &sd, nullptr));
  }
  *bytes = best + static_cast<size_t>(2) * kGridMax * ctd::kMaxN * sizeof(float);
  return CTD_OK;
}

ctd_status ctd_probe_cfem(const ctd_config* cfg, int d, double* omega, double* kband,
                          int* half_bandwidth_out) {
  ctd_status v = validate(cfg);
  if (v != CTD_OK) return v;
  if (d < 0 || d >= cfg->dim) return CTD_ERR_ARG;
  if (half_bandwidth_out) *half_bandwidth_out = half_bandwidth(cfg->s);
  if (ctd::build_cfem_1d(cfg->n[d], cfg->length[d], cfg->s, cfg->p, cfg->a, omega, kband) != 0)
    return CTD_ERR_ARG;
  return CTD_OK;
}

ctd_status ctd_probe_cfem_gauss(const ctd_config* cfg, int d, int q, double* x_q, double* omega_q, double* phi,
                                int* phi_col0, double* mband, double* mass_bounds) {
  ctd_status v = validate(cfg);
  if (v != CTD_OK) return v;
  if (d < 0 || d >= cfg->dim || q < 1 || q > ctd::kMaxGaussPoints) return CTD_ERR_ARG;
  if (ctd::build_cfem_gauss_1d(cfg->n[d], cfg->length[d], cfg->s, cfg->p, cfg->a, q, x_q, omega_q, phi, phi_col0,
                               mband, mass_bounds) != 0)
    return CTD_ERR_ARG;
  return CTD_OK;
}

ctd_status ctd_create(const ctd_config* cfg, void* workspace, size_t workspace_bytes,
                      void* cuda_stream, ctd_handle* out) {
  ctd_status v = validate(cfg);
  if (v != CTD_OK) return v;
  if (!out) return CTD_ERR_ARG;
  *out = nullptr;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CTD_ERR_WORKSPACE;
  size_t need = 0;
  ctd_workspace_size(cfg, &need);
  if (workspace_bytes < need) return CTD_ERR_WORKSPACE;

  ctd_ctx* h = new ctd_ctx();
  h->cfg = *cfg;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->has_modes = false;
  CTD_CUDA(h, cudaGetDevice(&h->device));
  int sms = 0, coop = 0;
  CTD_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  CTD_CUDA(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device));
  if (!coop) { ctd_status s = fail(h, CTD_ERR_UNSUPPORTED, "device lacks cooperative launch"); delete h; return s; }
  long long N = 1;
  for (int d = 0; d < cfg->dim; ++d) N *= cfg->n[d];
  int grid = cfg->grid_ctas > 0 ? cfg->grid_ctas
                                : static_cast<int>(std::min<long long>(sms, std::max<long long>(1, N / 16384)));
  grid = std::min(grid, sms);
  h->grid = grid;
  h->plan = make_plan(*cfg, grid);
  carve(*cfg, h->plan, workspace, &h->P, &h->X, h->kc_store, h->mc_store, &h->energy_part, &h->energy_gram,
        &h->stats_dev, &h->actd);
  h->P.vgrid = grid;   // each CTA sets its own rank in its shared-memory copy
  h->P.vrank = 0;

  StepParams& P = h->P;
  Extra& X = h->X;
  P.dim = cfg->dim;
  P.quad = h->plan.quad;
  P.actd_Mc = cfg->actd_Mc;
  P.quad_q = h->plan.quad ? cfg->quad_q : 1;
  P.Mcap = h->plan.Mcap;
  P.Kpad = h->plan.Kpad;
  P.precision = cfg->precision;
  P.c_t = 1.0 / cfg->dt + cfg->alpha * cfg->L;
  P.c_k = cfg->L * cfg->kappa;
  P.L = cfg->L;
  P.a0 = cfg->a0;
  {
    auto df = [](double v) {
      const float hi = static_cast<float>(v);
      return make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
    };
    P.ct_df = df(P.c_t);
    P.ck_df = df(P.c_k);
    P.L_df = df(P.L);
  }
  P.tol_als = cfg->tol_als;
  P.tol_enrich = cfg->tol_enrich;
  P.als_stall = cfg->als_stall_tol;
  P.reduced_tol = cfg->reduced_tol;
  P.nl_form = cfg->nonlinear_form;
  P.sep_q = h->plan.sep_q;
  P.contraction_form = cfg->contraction_form;
  P.I_max = cfg->I_max;
  P.M_max = cfg->M_max;
  P.fixed_als = cfg->fixed_als_iters;
  P.fixed_modes = cfg->fixed_modes;
  P.seed = cfg->seed;
  const double est = 4.0 * static_cast<double>(N) * cfg->M_max * 2.0 / 1.0e12;
  const double wait_s = cfg->wait_limit_s > 0.0 ? cfg->wait_limit_s : 1.0 + est;
  P.wait_ns = static_cast<unsigned long long>(wait_s * 1e9);
  for (int x = 0; x < cfg->dim; ++x) P.rchunks[x] = h->plan.rchunks[x];
  // Gershgorin bound of the generalised eigenvalues of (K, diag(omega)) per dimension
  for (int d = 0; d < cfg->dim; ++d) {
    const int n = cfg->n[d], w = 2 * h->plan.b[d] + 1;
    std::vector<double> om(n), kb(static_cast<size_t>(n) * w);
    ctd::build_cfem_1d(n, cfg->length[d], cfg->s, cfg->p, cfg->a, om.data(), kb.data());
    double g = 0.0;
    for (int i = 0; i < n; ++i) {
      double r = 0.0;
      for (int k = 0; k < w; ++k) r += std::fabs(kb[static_cast<size_t>(i) * w + k]);
      g = std::max(g, r / om[i]);
    }
    h->mu_max[d] = g * 1.000001;
    P.d[d].mu_max = static_cast<float>(h->mu_max[d]);
  }
  h->trace_dev = P.trace;
  P.trace = nullptr;

  // host C-FEM data and compressed stiffness per dimension
  for (int d = 0; d < cfg->dim; ++d) {
    const int n = cfg->n[d], b = h->plan.b[d], w = 2 * b + 1;
    h->omega[d].assign(n, 0.0);
    h->kband[d].assign(static_cast<size_t>(n) * w, 0.0);
    if (ctd::build_cfem_1d(n, cfg->length[d], cfg->s, cfg->p, cfg->a, h->omega[d].data(), h->kband[d].data()) != 0) {
      ctd_status s = fail(h, CTD_ERR_ARG, "C-FEM construction failed");
      delete h;
      return s;
    }
    CTD_CUDA(h, cudaMemcpyAsync(const_cast<double*>(P.d[d].omega), h->omega[d].data(), sizeof(double) * n,
                                cudaMemcpyHostToDevice, h->stream));
    CTD_CUDA(h, cudaMemcpyAsync(const_cast<double*>(P.d[d].kband), h->kband[d].data(),
                                sizeof(double) * n * w, cudaMemcpyHostToDevice, h->stream));
    // interior rows [2s+1, n-2-2s] share one stencil when the mesh is uniform
    const int s = cfg->s;
    int lead = 0, tail = 0;
    const std::vector<float2> kc = compress_band(h->kband[d], n, s, w, &lead, &tail);
    CTD_CUDA(h, cudaMemcpyAsync(h->kc_store[d], kc.data(), sizeof(float2) * kc.size(), cudaMemcpyHostToDevice,
                                h->stream));
    auto to_df = [](double v) {
      const float hi = static_cast<float>(v);
      return make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
    };
    ctd::KCompressed& k = X.kc[d];
    k.mrows = nullptr;
    k.mstencil = nullptr;
    k.mlead = k.mtail = 0;
    if (h->plan.quad) {
      // Gauss rule: points, weights, shape function values and the consistent mass band
      const int q = cfg->quad_q, nq = h->plan.nq[d], wphi = 2 * s + 2;
      std::vector<double> xq(nq), wq(nq), phi(static_cast<size_t>(nq) * wphi), mb(static_cast<size_t>(n) * w);
      std::vector<int> col0(nq);
      if (ctd::build_cfem_gauss_1d(n, cfg->length[d], s, cfg->p, cfg->a, q, xq.data(), wq.data(), phi.data(),
                                   col0.data(), mb.data(), nullptr) != 0) {
        ctd_status st = fail(h, CTD_ERR_ARG, "Gauss-rule construction failed");
        delete h;
        return st;
      }
      std::vector<float2> phid(static_cast<size_t>(nq) * ctd::kPhiW, make_float2(0.f, 0.f));
      for (int r = 0; r < nq; ++r)
        for (int j = 0; j < wphi; ++j) phid[static_cast<size_t>(r) * ctd::kPhiW + j] = to_df(phi[static_cast<size_t>(r) * wphi + j]);
      Dim& dd = P.d[d];
      CTD_CUDA(h, cudaMemcpyAsync(const_cast<double*>(dd.wq), wq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice,
                                  h->stream));
      CTD_CUDA(h, cudaMemcpyAsync(const_cast<float2*>(dd.phi), phid.data(), sizeof(float2) * phid.size(),
                                  cudaMemcpyHostToDevice, h->stream));
      CTD_CUDA(h, cudaMemcpyAsync(const_cast<int*>(dd.phi0), col0.data(), sizeof(int) * nq, cudaMemcpyHostToDevice,
                                  h->stream));
      CTD_CUDA(h, cudaMemcpyAsync(const_cast<double*>(dd.mband), mb.data(), sizeof(double) * mb.size(),
                                  cudaMemcpyHostToDevice, h->stream));
      int ml = 0, mt = 0;
      const std::vector<float2> mc = compress_band(mb, n, s, w, &ml, &mt);
      CTD_CUDA(h, cudaMemcpyAsync(h->mc_store[d], mc.data(), sizeof(float2) * mc.size(), cudaMemcpyHostToDevice,
                                  h->stream));
      CTD_CUDA(h, cudaStreamSynchronize(h->stream));   // the host vectors above are freed next
      k.mlead = ml;
      k.mtail = mt;
      k.mrows = h->mc_store[d];
      k.mstencil = h->mc_store[d] + static_cast<size_t>(ml + mt) * w;
      h->gphi[d] = phi;
      h->gcol0[d] = col0;
      h->gwq[d] = wq;
    }
    k.n = n;
    k.b = b;
    k.nlead = lead;
    k.ntail = tail;
    k.rows = h->kc_store[d];
    k.stencil = h->kc_store[d] + static_cast<size_t>(lead + tail) * w;
    k.omega_in = to_df(h->omega[d][n / 2]);
    k.omega_end = to_df(h->omega[d][0]);
    k.inv_omega_in = static_cast<float>(1.0 / h->omega[d][n / 2]);
    k.inv_omega_end = static_cast<float>(1.0 / h->omega[d][0]);
  }
  // shared memory: fixed part + per-phase arena; solver factors join the arena if they fit
  {
    int n_max = 0;
    size_t crf = 0, l0f = 0;
    for (int d = 0; d < cfg->dim; ++d) {
      n_max = std::max(n_max, cfg->n[d]);
      crf = std::max(crf, ctd::cr_floats(cfg->n[d], h->plan.b[d]));
      l0f = std::max(l0f, ctd::l0_smem_floats(cfg->n[d], h->plan.b[d]));
    }
    int optin = 0;
    CTD_CUDA(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    const size_t fixed = ctd::step_smem_fixed_bytes();
    const size_t margin = 1024 + 2048;   // arena alignment + static shared variables
    P.n_max = n_max;
    // Chebyshev unless its worst-case iteration count (smallest beta = c_t / c_k) is large
    int worst_its = 0;
    for (int d = 0; d < cfg->dim; ++d)
      worst_its = std::max(worst_its, ctd::cheb_iterations(static_cast<float>(P.c_t), static_cast<float>(P.c_k),
                                                           static_cast<float>(h->mu_max[d]), 2.384185791015625e-07f));
    const size_t chf = ctd::cheb_floats(n_max);
    bool cheb_split = true;   // every dimension has a row split for the Chebyshev CTA
    for (int d = 0; d < cfg->dim; ++d) {
      ctd::ChebLayout lay;
      if (!ctd::cheb_layout(cfg->n[d], X.kc[d].nlead, X.kc[d].ntail, X.kc[d].b, ctd::kThreads - 32, lay))
        cheb_split = false;
    }
    // the Chebyshev split is built around the nodal rule's diagonal mass; the Gauss rule's
    // consistent mass takes block cyclic reduction
    if (!h->plan.quad && cheb_split && worst_its <= 200 &&
        fixed + ctd::step_arena_bytes(n_max, chf, 3) + margin <= static_cast<size_t>(optin))
      P.solver_mode = 3;
    else if (fixed + ctd::step_arena_bytes(n_max, crf, 0) + margin <= static_cast<size_t>(optin)) P.solver_mode = 0;
    else if (fixed + ctd::step_arena_bytes(n_max, l0f, 1) + margin <= static_cast<size_t>(optin)) P.solver_mode = 1;
    else P.solver_mode = 2;
    const size_t used = P.solver_mode == 3 ? chf : (P.solver_mode == 0 ? crf : l0f);
    size_t need = fixed + ctd::step_arena_bytes(n_max, used, P.solver_mode) + 1024;
    if (cfg->precision != CTD_PREC_FP64) {
      const int chunks = ctd::tc_nimg(cfg->precision) * h->plan.Kpad / ctd::kTcChunkElems;
      int stages = 4;
      for (; stages >= 1; --stages) {
        size_t tcb = 0;
        for (int x = 0; x < cfg->dim; ++x) {
          const ctd::TcDir& td = h->plan.dirs[x];
          const int wl = td.mid < 0 ? td.ncols_pad : td.n_last_pad;
          const int wm = td.mid < 0 ? 0 : h->plan.nq[td.mid];
          tcb = std::max(tcb, ctd::tc_layout(chunks, stages, wl, wm).total);
        }
        if (fixed + 1024 + tcb + 1024 <= static_cast<size_t>(optin)) {
          need = std::max(need, fixed + 1024 + tcb);
          break;
        }
      }
      if (stages < 1) { ctd_status s = fail(h, CTD_ERR_UNSUPPORTED, "tensor-core tiles exceed shared memory"); delete h; return s; }
      X.tc_stages = stages;
    }
    // the tensor-core path allocates all 512 TMEM columns of the SM: more than half the shared
    // memory keeps it at one CTA per SM, so no CTA waits for another's columns
    if (cfg->precision != CTD_PREC_FP64) need = std::max(need, static_cast<size_t>(optin) / 2 + 1024);
    if (cfg->precision != CTD_PREC_FP64 && cfg->reduced_tol > 0.0) {
      // block classification stages every dimension's factor rows of a block
      const size_t cls = fixed + 1024 + static_cast<size_t>(cfg->dim) * h->plan.Mcap * ctd::kTcM * sizeof(float) + 1024;
      if (cls > static_cast<size_t>(optin)) {
        ctd_status s = fail(h, CTD_ERR_UNSUPPORTED, "reduced-domain classification exceeds shared memory");
        delete h;
        return s;
      }
      need = std::max(need, cls);
    }
    P.smem_bytes = static_cast<int>(need);
  }
  if (cfg->actd_Mc > 0) {
    // the omega and band uploads above read host vectors that live in the handle
    const double* kb[3] = {nullptr, nullptr, nullptr};
    const double* om[3] = {nullptr, nullptr, nullptr};
    for (int d = 0; d < cfg->dim; ++d) {
      kb[d] = h->kband[d].data();
      om[d] = h->omega[d].data();
    }
    const char* msg = "";
    const int rc = ctd::actd_setup(h->actd, P, kb, om, h->stream, &msg);
    if (rc != 0) {
      ctd_status s = fail(h, static_cast<ctd_status>(rc), msg);
      g_create_err = msg;
      ctd::actd_release(h->actd);
      delete h;
      return s;
    }
  }
  InstState st{};
  CTD_CUDA(h, cudaMemcpyAsync(P.st, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = h;
  return CTD_OK;
}

ctd_status ctd_set_initial_modes(ctd_handle h, int rank, const double* const* modes, int on_device,
                                 long long first_step) {
  if (!h) return CTD_ERR_ARG;
  if (rank < 0 || rank > h->cfg.M_max || (rank > 0 && !modes)) return fail(h, CTD_ERR_ARG, "bad rank or modes");
  for (int d = 0; d < h->cfg.dim; ++d) {
    const int n = h->cfg.n[d];
    if (rank == 0) break;
    if (!modes[d]) return fail(h, CTD_ERR_ARG, "null factor array");
    float2* dst = h->P.d[d].bank[0];
    if (on_device) {
      CTD_CUDA(h, ctd::launch_modes_from_fp64(dst, modes[d], static_cast<long long>(rank) * n, h->stream));
    } else {
      std::vector<float2> tmp(static_cast<size_t>(rank) * n);
      for (size_t t = 0; t < tmp.size(); ++t) {
        const double v = modes[d][t];
        if (!std::isfinite(v)) return fail(h, CTD_ERR_NONFINITE, "non-finite initial mode entry");
        const float hi = static_cast<float>(v);
        tmp[t] = make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
      }
      CTD_CUDA(h, cudaMemcpyAsync(dst, tmp.data(), sizeof(float2) * tmp.size(), cudaMemcpyHostToDevice, h->stream));
      CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    }
  }
  InstState st{};
  st.Mk = rank;
  st.bank = 0;
  st.step = first_step;
  CTD_CUDA(h, cudaMemcpyAsync(h->P.st, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  h->has_modes = true;
  return CTD_OK;
}

static ctd_status read_state(ctd_handle h, InstState* st) {
  CTD_CUDA(h, cudaMemcpyAsync(st, h->P.st, sizeof(InstState), cudaMemcpyDeviceToHost, h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  return CTD_OK;
}

ctd_status ctd_step(ctd_handle h, int nsteps, ctd_step_stats* stats) {
  if (!h || nsteps < 0) return CTD_ERR_ARG;
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "ctd_set_initial_modes has not been called");
  ctd_status worst = CTD_OK;
  std::vector<StepStatsDev> rec;
  int done = 0;
  // adaptive CTD: one step at a time, the switch decision read back after each
  const bool actd = h->P.actd_Mc > 0;
  while (done < nsteps) {
    const int batch = actd ? 1 : std::min(nsteps - done, kStatsCap);
    for (int k = 0; k < batch; ++k) {
      h->P.stats = h->stats_dev + k;
      CTD_CUDA(h, cudaMemsetAsync(h->P.barrier, 0, sizeof(unsigned), h->stream));
      CTD_CUDA(h, h->P.nl_form == CTD_NONLINEAR_SEPARATED ? ctd::launch_step_sep(h->P, h->X, h->grid, h->stream)
                                                         : ctd::launch_step(h->P, h->X, h->grid, h->stream));
    }
    if (actd) {
      InstState st;
      ctd_status rs = read_state(h, &st);
      if (rs != CTD_OK) return rs;
      if (st.status) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "device status %d at wait %d", st.status, st.err_info);
        return fail(h, status_from_bits(st.status), buf);
      }
      if (st.switched) {
        // the step needs more than M_c modes: solve it on the full grid from u^k
        const char* msg = "";
        const int rc = ctd::actd_cfe_step(h->actd, h->P, st.grid, st.bank, st.Mk, h->stream, &msg);
        if (rc != 0) return fail(h, static_cast<ctd_status>(rc), msg);
        st.grid = 1;
        st.Mk = 0;
        st.switched = 0;
        CTD_CUDA(h, cudaMemcpyAsync(h->P.st, &st, sizeof(st), cudaMemcpyHostToDevice, h->stream));
        CTD_CUDA(h, cudaStreamSynchronize(h->stream));
      }
    }
    if (stats) {
      rec.resize(batch);
      CTD_CUDA(h, cudaMemcpyAsync(rec.data(), h->stats_dev, sizeof(StepStatsDev) * batch, cudaMemcpyDeviceToHost,
                                  h->stream));
      InstState st;
      ctd_status rs = read_state(h, &st);
      if (rs != CTD_OK) return rs;
      const ctd_status es = status_from_bits(st.status);
      for (int k = 0; k < batch; ++k) {
        ctd_step_stats& o = stats[done + k];
        o.modes = rec[k].modes;
        o.als_sweeps = rec[k].als_sweeps;
        o.als_sweeps_max = rec[k].als_sweeps_max;
        o.capped = rec[k].capped;
        o.not_converged = rec[k].not_converged;
        o.als_stalled = rec[k].als_stalled;
        o.als_sweeps_committed = rec[k].als_sweeps_committed;
        o.actd_switched = rec[k].actd_switched;
        o.cube_form = rec[k].cube_form;
        o.status = es != CTD_OK ? es : (o.capped ? CTD_STATUS_CAPPED : (o.not_converged ? CTD_STATUS_ALS_NOT_CONVERGED : CTD_OK));
        if (o.status < 0) worst = static_cast<ctd_status>(o.status);
        else if (worst >= 0 && o.status > worst) worst = static_cast<ctd_status>(o.status);
      }
      if (es != CTD_OK) {
        char buf[128];
        std::snprintf(buf, sizeof buf, "device status %d at wait %d", st.status, st.err_info);
        return fail(h, es, buf);
      }
    }
    done += batch;
  }
  if (!stats) CTD_CUDA(h, cudaGetLastError());
  return worst;
}

ctd_status ctd_batch_workspace_size(int count, size_t* bytes) {
  if (count < 1 || !bytes) return CTD_ERR_ARG;
  *bytes = (sizeof(ctd::BatchEntry) * static_cast<size_t>(count) + 255) / 256 * 256 +
           (sizeof(int) * static_cast<size_t>(count) + 255) / 256 * 256;
  return CTD_OK;
}

ctd_status ctd_step_batch(const ctd_handle* handles, int count, int nsteps, void* workspace,
                          size_t workspace_bytes, void* cuda_stream, ctd_step_stats* stats) {
  if (!handles || count < 1 || nsteps < 0) return CTD_ERR_ARG;
  size_t need = 0;
  ctd_batch_workspace_size(count, &need);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CTD_ERR_WORKSPACE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CTD_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    ctd_ctx* h = handles[i];
    if (!h) return CTD_ERR_ARG;
    if (!h->has_modes) return fail(h, CTD_ERR_STATE, "ctd_set_initial_modes has not been called");
    if (h->device != dev) return fail(h, CTD_ERR_STATE, "instance on another device");
    if (h->P.nl_form != CTD_NONLINEAR_GRID)
      return fail(h, CTD_ERR_UNSUPPORTED, "batched steps integrate the nonlinear term over the grid only");
    if (h->P.quad) return fail(h, CTD_ERR_UNSUPPORTED, "batched steps take the nodal rule only");
    if (h->P.actd_Mc > 0) return fail(h, CTD_ERR_UNSUPPORTED, "batched steps do not switch to the full grid");
  }
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // one entry per instance; the largest instances start first
  std::vector<ctd::BatchEntry> entries(count);
  std::vector<int> order(count);
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    ctd_ctx* h = handles[i];
    std::memset(&entries[i], 0, sizeof(ctd::BatchEntry));
    entries[i].P = h->P;
    entries[i].P.stats = h->stats_dev;
    entries[i].P.trace = nullptr;
    entries[i].X = h->X;
    smem = std::max(smem, static_cast<size_t>(h->P.smem_bytes));
    order[i] = i;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return handles[a]->plan.N > handles[b]->plan.N; });
  auto* dev_entries = static_cast<ctd::BatchEntry*>(workspace);
  int* dev_order = reinterpret_cast<int*>(static_cast<char*>(workspace) +
                                          (sizeof(ctd::BatchEntry) * static_cast<size_t>(count) + 255) / 256 * 256);
  ctd_ctx* h0 = handles[0];
  CTD_CUDA(h0, cudaMemcpyAsync(dev_entries, entries.data(), sizeof(ctd::BatchEntry) * count, cudaMemcpyHostToDevice,
                               stream));
  CTD_CUDA(h0, cudaMemcpyAsync(dev_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, stream));
  ctd_status worst = CTD_OK;
  std::vector<StepStatsDev> rec;
  int done = 0;
  while (done < nsteps) {
    const int batch = std::min(nsteps - done, kStatsCap);
    for (int k = 0; k < batch; ++k) CTD_CUDA(h0, ctd::launch_batch_step(dev_entries, dev_order, count, k, smem, stream));
    if (stats) {
      CTD_CUDA(h0, cudaStreamSynchronize(stream));
      rec.resize(batch);
      for (int i = 0; i < count; ++i) {
        ctd_ctx* h = handles[i];
        CTD_CUDA(h, cudaMemcpy(rec.data(), h->stats_dev, sizeof(StepStatsDev) * batch, cudaMemcpyDeviceToHost));
        InstState st;
        CTD_CUDA(h, cudaMemcpy(&st, h->P.st, sizeof(InstState), cudaMemcpyDeviceToHost));
        const ctd_status es = status_from_bits(st.status);
        for (int k = 0; k < batch; ++k) {
          ctd_step_stats& o = stats[static_cast<size_t>(i) * nsteps + done + k];
          o.modes = rec[k].modes;
          o.als_sweeps = rec[k].als_sweeps;
          o.als_sweeps_max = rec[k].als_sweeps_max;
          o.capped = rec[k].capped;
          o.not_converged = rec[k].not_converged;
          o.als_stalled = rec[k].als_stalled;
          o.als_sweeps_committed = rec[k].als_sweeps_committed;
          o.actd_switched = rec[k].actd_switched;
          o.cube_form = rec[k].cube_form;
          o.status = es != CTD_OK ? es : (o.capped ? CTD_STATUS_CAPPED : (o.not_converged ? CTD_STATUS_ALS_NOT_CONVERGED : CTD_OK));
          if (o.status < 0) worst = static_cast<ctd_status>(o.status);
          else if (worst >= 0 && o.status > worst) worst = static_cast<ctd_status>(o.status);
        }
        if (es != CTD_OK) fail(h, es, "device status set");
      }
      if (worst < 0) return worst;
    }
    done += batch;
  }
  if (!stats) CTD_CUDA(h0, cudaGetLastError());
  return worst;
}

ctd_status ctd_energy(ctd_handle h, double* energy) {
  if (!h || !energy) return CTD_ERR_ARG;
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.status) return fail(h, status_from_bits(st.status), "device status set");
  const int Mk = st.Mk, D = h->cfg.dim;
  int sms = 0;
  CTD_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const int eg = std::min(1024, 4 * sms);
  if (st.grid) {
    // adaptive CTD: the field is the full-grid array
    CTD_CUDA(h, ctd::launch_energy_grid(h->P, h->P.U, h->energy_part, eg, h->stream));
    std::vector<double> part(eg);
    CTD_CUDA(h, cudaMemcpyAsync(part.data(), h->energy_part, sizeof(double) * eg, cudaMemcpyDeviceToHost, h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    double e = 0.0;
    for (int g = 0; g < eg; ++g) e += part[g];
    *energy = e;
    return CTD_OK;
  }
  CTD_CUDA(h, ctd::launch_convert_modes(h->P, h->X, st.bank, Mk, h->stream));
  CTD_CUDA(h, ctd::launch_energy_bulk(h->P, h->X, Mk, h->energy_part, eg, h->stream));
  CTD_CUDA(h, ctd::launch_energy_gram(h->P, h->X, Mk, h->energy_gram, h->stream));
  std::vector<double> part(eg), gram(static_cast<size_t>(D) * 2 * Mk * Mk);
  CTD_CUDA(h, cudaMemcpyAsync(part.data(), h->energy_part, sizeof(double) * eg, cudaMemcpyDeviceToHost, h->stream));
  if (Mk)
    CTD_CUDA(h, cudaMemcpyAsync(gram.data(), h->energy_gram, sizeof(double) * gram.size(), cudaMemcpyDeviceToHost,
                                h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  double bulk = 0.0;
  for (int g = 0; g < eg; ++g) bulk += part[g];
  double grad = 0.0;
  for (int a = 0; a < Mk; ++a)
    for (int c = 0; c < Mk; ++c)
      for (int d = 0; d < D; ++d) {
        double t = gram[(static_cast<size_t>(d) * 2 + 1) * Mk * Mk + a * Mk + c];
        for (int e = 0; e < D; ++e)
          if (e != d) t *= gram[(static_cast<size_t>(e) * 2 + 0) * Mk * Mk + a * Mk + c];
        grad += t;
      }
  *energy = bulk + 0.5 * h->cfg.kappa * grad;
  return CTD_OK;
}

ctd_status ctd_get_modes(ctd_handle h, int capacity, int* rank, double* const* modes_out, int on_device) {
  if (!h || !rank) return CTD_ERR_ARG;
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.grid) {
    *rank = 0;
    return fail(h, CTD_ERR_STATE, "the field is held on the full grid (read it with ctd_get_field)");
  }
  *rank = st.Mk;
  if (capacity < st.Mk) return fail(h, CTD_ERR_ARG, "capacity below rank");
  if (st.Mk == 0) return CTD_OK;
  if (!modes_out) return CTD_ERR_ARG;
  for (int d = 0; d < h->cfg.dim; ++d) {
    const int n = h->cfg.n[d];
    if (!modes_out[d]) return fail(h, CTD_ERR_ARG, "null output array");
    const float2* src = h->P.d[d].bank[st.bank];
    if (on_device) {
      CTD_CUDA(h, ctd::launch_modes_to_fp64(modes_out[d], src, static_cast<long long>(st.Mk) * n, h->stream));
    } else {
      std::vector<float2> tmp(static_cast<size_t>(st.Mk) * n);
      CTD_CUDA(h, cudaMemcpyAsync(tmp.data(), src, sizeof(float2) * tmp.size(), cudaMemcpyDeviceToHost, h->stream));
      CTD_CUDA(h, cudaStreamSynchronize(h->stream));
      for (size_t t = 0; t < tmp.size(); ++t)
        modes_out[d][t] = static_cast<double>(tmp[t].x) + static_cast<double>(tmp[t].y);
    }
  }
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  return CTD_OK;
}

ctd_status ctd_get_field(ctd_handle h, double* out, int on_device) {
  if (!h || !out) return CTD_ERR_ARG;
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  size_t nodes = 1;   // the field's values at the nodes (also under the Gauss rule)
  for (int d = 0; d < h->cfg.dim; ++d) nodes *= static_cast<size_t>(h->cfg.n[d]);
  if (st.grid) {
    CTD_CUDA(h, cudaMemcpyAsync(out, h->P.U, sizeof(double) * nodes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    return CTD_OK;
  }
  if (on_device) {
    CTD_CUDA(h, ctd::launch_field_from_modes(h->P, st.bank, st.Mk, out, h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    return CTD_OK;
  }
  // host output: rebuild from the factors on the host
  const int D = h->cfg.dim, Mk = st.Mk;
  std::vector<std::vector<double>> f(D);
  for (int d = 0; d < D; ++d) {
    const int n = h->cfg.n[d];
    std::vector<float2> tmp(static_cast<size_t>(Mk) * n);
    if (Mk)
      CTD_CUDA(h, cudaMemcpyAsync(tmp.data(), h->P.d[d].bank[st.bank], sizeof(float2) * tmp.size(),
                                  cudaMemcpyDeviceToHost, h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    f[d].resize(tmp.size());
    for (size_t t = 0; t < tmp.size(); ++t) f[d][t] = static_cast<double>(tmp[t].x) + static_cast<double>(tmp[t].y);
  }
  const int n0 = h->cfg.n[0], n1 = h->cfg.n[1], n2 = D == 3 ? h->cfg.n[2] : 1;
  for (int i = 0; i < n0; ++i)
    for (int j = 0; j < n1; ++j)
      for (int l = 0; l < n2; ++l) {
        double u = 0.0;
        for (int m = 0; m < Mk; ++m) {
          double t = f[0][static_cast<size_t>(m) * n0 + i] * f[1][static_cast<size_t>(m) * n1 + j];
          if (D == 3) t *= f[2][static_cast<size_t>(m) * n2 + l];
          u += t;
        }
        out[(static_cast<size_t>(i) * n1 + j) * n2 + l] = u;
      }
  return CTD_OK;
}

void ctd_destroy(ctd_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  ctd::actd_release(h->actd);
  delete h;
}

ctd_status ctd_probe_contract(ctd_handle h, int x, const double* const* v, double* out) {
  if (!h || !v || !out || x < 0 || x >= h->cfg.dim) return CTD_ERR_ARG;
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  for (int d = 0; d < h->cfg.dim; ++d) {
    if (d == x) continue;
    if (!v[d]) return CTD_ERR_ARG;
    const int n = h->cfg.n[d];
    std::vector<float2> tmp(n);
    for (int i = 0; i < n; ++i) {
      const float hi = static_cast<float>(v[d][i]);
      tmp[i] = make_float2(hi, static_cast<float>(v[d][i] - static_cast<double>(hi)));
    }
    CTD_CUDA(h, cudaMemcpyAsync(h->P.d[d].v, tmp.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  CTD_CUDA(h, cudaMemsetAsync(h->P.barrier, 0, sizeof(unsigned), h->stream));
  // partial slots of CTAs without a tile in a row block are not written: start from zero
  CTD_CUDA(h, cudaMemsetAsync(h->X.rpart_tc, 0, sizeof(double) * std::max<size_t>(1, h->plan.rpart_tc_len), h->stream));
  CTD_CUDA(h, ctd::launch_probe_contract(h->P, h->X, h->grid, x, nullptr, h->stream));
  const int n = h->cfg.n[x], nq = h->plan.nq[x];
  std::vector<double> rq(nq);   // weighted sums at the points of direction x (the nodes, nodal rule)
  if (h->cfg.precision == CTD_PREC_FP64) {
    const int C = h->plan.rchunks[x];
    std::vector<double> part(static_cast<size_t>(nq) * C);
    CTD_CUDA(h, cudaMemcpyAsync(part.data(), h->P.rpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                                h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < nq; ++i) {
      double r = 0.0;
      for (int k = 0; k < C; ++k) r += part[static_cast<size_t>(i) * C + k];
      rq[i] = r;
    }
  } else {
    const ctd::TcDir& td = h->plan.dirs[x];
    std::vector<double> part(static_cast<size_t>(nq) * td.cmax);
    CTD_CUDA(h, cudaMemcpyAsync(part.data(), h->X.rpart_tc, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                                h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    const long long T = static_cast<long long>(td.nrb) * td.ntc;
    for (int i = 0; i < nq; ++i) {
      const int rb = i / ctd::kTcM;
      const int c0 = ctd::tile_owner(T, h->grid, static_cast<long long>(rb) * td.ntc);
      const int c1 = ctd::tile_owner(T, h->grid, static_cast<long long>(rb) * td.ntc + td.ntc - 1);
      double r = 0.0;
      for (int k = 0; k <= c1 - c0; ++k) r += part[static_cast<size_t>(i) * td.cmax + k];
      rq[i] = r;
    }
  }
  if (h->plan.quad) {
    // Gauss rule: Phi_x^T of the point sums
    const int wphi = 2 * h->cfg.s + 2;
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (int r = 0; r < nq; ++r)
      for (int k = 0; k < wphi; ++k) {
        const int i = h->gcol0[x][r] + k;
        if (i < n) out[i] += h->gphi[x][static_cast<size_t>(r) * wphi + k] * h->gwq[x][r] * rq[r];
      }
  } else {
    for (int i = 0; i < n; ++i) out[i] = rq[i];
  }
  if (h->cfg.precision != CTD_PREC_FP64) {
    // tensor-core partials: without the factor 4 a0, and in the cube form without the linear
    // part, which the probe kernel left in P.rpart
    int cube = 0;
    CTD_CUDA(h, cudaMemcpyAsync(&cube, h->X.ctrl + 2, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
    if (cube) {
      std::vector<double> lin(n);
      CTD_CUDA(h, cudaMemcpyAsync(lin.data(), h->P.rpart, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
      CTD_CUDA(h, cudaStreamSynchronize(h->stream));
      for (int i = 0; i < n; ++i) out[i] -= lin[i];
    }
    for (int i = 0; i < n; ++i) out[i] *= 4.0 * h->cfg.a0;
  }
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.status) return fail(h, status_from_bits(st.status), "device status set");
  return CTD_OK;
}

ctd_status ctd_probe_reconstruct(ctd_handle h, int x, float* out, void* scratch, size_t scratch_bytes) {
  if (!h || !out || x < 0 || x >= h->cfg.dim) return CTD_ERR_ARG;
  if (h->cfg.precision == CTD_PREC_FP64) return fail(h, CTD_ERR_UNSUPPORTED, "tensor-core path only");
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  const ctd::TcDir& td = h->plan.dirs[x];
  const size_t need = static_cast<size_t>(h->plan.n_pad[x]) * td.ncols_pad * sizeof(float);
  if (!scratch || scratch_bytes < need) return fail(h, CTD_ERR_WORKSPACE, "scratch too small");
  // weights are irrelevant for the dump; keep v finite
  for (int d = 0; d < h->cfg.dim; ++d) {
    std::vector<float2> ones(h->cfg.n[d], make_float2(1.f, 0.f));
    CTD_CUDA(h, cudaMemcpyAsync(h->P.d[d].v, ones.data(), sizeof(float2) * ones.size(), cudaMemcpyHostToDevice,
                                h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  CTD_CUDA(h, cudaMemsetAsync(scratch, 0, need, h->stream));
  CTD_CUDA(h, cudaMemsetAsync(h->P.barrier, 0, sizeof(unsigned), h->stream));
  CTD_CUDA(h, ctd::launch_probe_contract(h->P, h->X, h->grid, x, static_cast<float*>(scratch), h->stream));
  CTD_CUDA(h, cudaMemcpyAsync(out, scratch, need, cudaMemcpyDeviceToHost, h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.status) return fail(h, status_from_bits(st.status), "device status set");
  return CTD_OK;
}

ctd_status ctd_probe_reconstruct_noalloc(ctd_handle h, int x, float* out) {
  if (!h || !out || x < 0 || x >= h->cfg.dim) return CTD_ERR_ARG;
  if (h->cfg.precision == CTD_PREC_FP64) return fail(h, CTD_ERR_UNSUPPORTED, "tensor-core path only");
  const ctd::TcDir& td = h->plan.dirs[x];
  const size_t need = static_cast<size_t>(h->plan.n_pad[x]) * td.ncols_pad * sizeof(float);
  if (need > CTD_RECONSTRUCT_STATIC_BYTES) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "tile grid of %zu bytes exceeds the %zu-byte static dump array", need,
                  static_cast<size_t>(CTD_RECONSTRUCT_STATIC_BYTES));
    return fail(h, CTD_ERR_WORKSPACE, buf);
  }
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  int cur = -1;
  CTD_CUDA(h, cudaGetDevice(&cur));
  if (cur != h->device) return fail(h, CTD_ERR_STATE, "current device is not the handle's");
  void* scratch = nullptr;
  CTD_CUDA(h, static_dump_address(cur, &scratch));
  for (int d = 0; d < h->cfg.dim; ++d) {
    std::vector<float2> ones(h->cfg.n[d], make_float2(1.f, 0.f));
    CTD_CUDA(h, cudaMemcpyAsync(h->P.d[d].v, ones.data(), sizeof(float2) * ones.size(), cudaMemcpyHostToDevice,
                                h->stream));
    CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  CTD_CUDA(h, cudaMemsetAsync(scratch, 0, need, h->stream));
  CTD_CUDA(h, cudaMemsetAsync(h->P.barrier, 0, sizeof(unsigned), h->stream));
  CTD_CUDA(h, ctd::launch_probe_contract(h->P, h->X, h->grid, x, static_cast<float*>(scratch), h->stream));
  CTD_CUDA(h, cudaMemcpyAsync(out, scratch, need, cudaMemcpyDeviceToHost, h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.status) return fail(h, status_from_bits(st.status), "device status set");
  return CTD_OK;
}

ctd_status ctd_probe_trace(ctd_handle h, int enable, double* seconds, int nslots) {
  if (!h || nslots < 0) return CTD_ERR_ARG;
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  if (seconds && nslots > 0) {
    unsigned long long t[ctd::kTrSlots];
    CTD_CUDA(h, cudaMemcpy(t, h->trace_dev, sizeof(t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < nslots; ++i) seconds[i] = i < ctd::kTrSlots ? 1e-9 * static_cast<double>(t[i]) : 0.0;
  }
  CTD_CUDA(h, cudaMemset(h->trace_dev, 0, sizeof(unsigned long long) * ctd::kTrSlots));
  h->P.trace = enable ? h->trace_dev : nullptr;
  return CTD_OK;
}

ctd_status ctd_probe_solve(ctd_handle h, int x, double alpha1, double alpha2, const double* q, double* y) {
  if (!h || !q || !y || x < 0 || x >= h->cfg.dim) return CTD_ERR_ARG;
  const int n = h->cfg.n[x];
  std::vector<float2> tmp(n);
  for (int i = 0; i < n; ++i) {
    const float hi = static_cast<float>(q[i]);
    tmp[i] = make_float2(hi, static_cast<float>(q[i] - static_cast<double>(hi)));
  }
  CTD_CUDA(h, cudaMemcpyAsync(h->P.Q, tmp.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, h->stream));
  CTD_CUDA(h, ctd::launch_probe_solve(h->P, h->X, x, alpha1, alpha2, h->stream));
  CTD_CUDA(h, cudaMemcpyAsync(tmp.data(), h->P.d[x].v, sizeof(float2) * n, cudaMemcpyDeviceToHost, h->stream));
  int flag = 0;
  CTD_CUDA(h, cudaMemcpyAsync(&flag, h->X.ctrl + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < n; ++i) y[i] = static_cast<double>(tmp[i].x) + static_cast<double>(tmp[i].y);
  if (flag) return fail(h, CTD_ERR_NONFINITE, "solver reported a failed pivot or non-finite value");
  return CTD_OK;
}

}  // extern "C"

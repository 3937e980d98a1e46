// C ABI of the CTD solver (declared in include/ctd.h): workspace layout, handle, launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctd.h"
#include "cfem_host.h"
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
  int D, n[3], b[3], n_pad[3], Mcap, Kpad, grid, rchunks[3];
  long long N;
  size_t rpart_len;
};

int half_bandwidth(int s) { return 2 * s + 1; }

int chunks_for(const ctd_config& c, int x, int grid) {
  const int D = c.dim, nc = c.n[x];
  const long long tw = static_cast<long long>(grid) * ctd::kWarps;
  long long C;
  if (x == D - 1) {
    long long rows = 1;
    for (int d = 0; d < D; ++d)
      if (d != x) rows *= c.n[d];
    const long long cblocks = (nc + 31) / 32;
    C = std::min<long long>(rows, std::max<long long>(1, (4 * tw + cblocks - 1) / cblocks));
  } else {
    const int extent = (D == 2) ? c.n[1] : (x == 0 ? c.n[1] : c.n[0]);
    C = std::min<long long>(extent, std::max<long long>(1, (4 * tw + nc - 1) / nc));
  }
  return static_cast<int>(C);
}

Plan make_plan(const ctd_config& c, int grid) {
  Plan p{};
  p.D = c.dim;
  p.N = 1;
  for (int d = 0; d < c.dim; ++d) {
    p.n[d] = c.n[d];
    p.b[d] = half_bandwidth(c.s);
    p.n_pad[d] = (c.n[d] + ctd::kTileRows - 1) / ctd::kTileRows * ctd::kTileRows;
    p.N *= c.n[d];
  }
  p.Mcap = c.M_max;
  p.Kpad = (c.M_max + 63) / 64 * 64;
  p.grid = grid;
  p.rpart_len = 0;
  for (int x = 0; x < c.dim; ++x) {
    p.rchunks[x] = chunks_for(c, x, grid);
    p.rpart_len = std::max(p.rpart_len, static_cast<size_t>(c.n[x]) * p.rchunks[x]);
  }
  return p;
}

// Lay out every workspace piece; fills P and X pointers when base != null.
size_t carve(const ctd_config& c, const Plan& pl, void* base, StepParams* P, Extra* X,
             float2** kc_store, double** energy_part, double** energy_gram, StepStatsDev** stats) {
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
    dd.op = nullptr;
    kc_store[d] = cv.take<float2>(static_cast<size_t>(n + 1) * w);
    x.Af[d] = cv.take<double>(static_cast<size_t>(pl.Mcap) * n);
  }
  int nmax = 0;
  for (int d = 0; d < D; ++d) nmax = std::max(nmax, pl.n[d]);
  const int spd = ctd::slots_per_dim(pl.Mcap);
  const int nslots = std::max((D - 1) * spd, D * 6);
  p.gram = cv.take<float2>(static_cast<size_t>(nslots) * Gs);
  p.rpart = cv.take<double>(pl.rpart_len);
  x.rpart32 = cv.take<float>(pl.rpart_len);
  p.Q = cv.take<float2>(ctd::kMaxN);
  size_t crf = 0;
  for (int d = 0; d < D; ++d) crf = std::max(crf, ctd::cr_floats(pl.n[d], pl.b[d]));
  p.solver = cv.take<float>(crf);
  p.W = (c.precision == CTD_PREC_FP64) ? cv.take<double>(static_cast<size_t>(pl.N)) : nullptr;
  p.barrier = cv.take<unsigned>(64);
  p.st = cv.take<InstState>(1);
  x.maxpart = cv.take<double>(static_cast<size_t>(ctd::kMaxDim) * Gs);
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
    case CTD_STATUS_ALS_NOT_CONVERGED: return "a mode reached I_max sweeps without meeting tol_als";
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
  if (c->fixed_als_iters < 0 || c->fixed_modes < 0 || c->fixed_modes > c->M_max) return CTD_ERR_ARG;
  if (c->precision != CTD_PREC_FP64 && c->precision != CTD_PREC_SPLIT_BF16) return CTD_ERR_ARG;
  if (c->grid_ctas > kGridMax) return CTD_ERR_ARG;
  return CTD_OK;
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
  double* energy_part;
  double* energy_gram;
  StepStatsDev* stats_dev;
  std::vector<double> omega[3], kband[3];
  bool has_modes;
  std::string err;
};

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

static ctd_status status_from_bits(int bits) {
  if (bits & ctd::kErrTimeout) return CTD_ERR_TIMEOUT;
  if (bits & (ctd::kErrNonfinite | ctd::kErrSolve)) return CTD_ERR_NONFINITE;
  return CTD_OK;
}

extern "C" {

const char* ctd_status_string(int status) { return status_text(status); }

const char* ctd_last_error(ctd_handle h) {
  if (!h) return "no handle";
  return h->err.c_str();
}

ctd_status ctd_workspace_size(const ctd_config* cfg, size_t* bytes) {
  ctd_status v = validate(cfg);
  if (v != CTD_OK) return v;
  if (!bytes) return CTD_ERR_ARG;
  if (cfg->precision == CTD_PREC_SPLIT_BF16) return CTD_ERR_UNSUPPORTED;
  float2* kc[3];
  double *ep, *eg;
  StepStatsDev* sd;
  const Plan pl = make_plan(*cfg, kGridMax);
  *bytes = carve(*cfg, pl, nullptr, nullptr, nullptr, kc, &ep, &eg, &sd);
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

ctd_status ctd_create(const ctd_config* cfg, void* workspace, size_t workspace_bytes,
                      void* cuda_stream, ctd_handle* out) {
  ctd_status v = validate(cfg);
  if (v != CTD_OK) return v;
  if (!out) return CTD_ERR_ARG;
  *out = nullptr;
  if (cfg->precision == CTD_PREC_SPLIT_BF16) return CTD_ERR_UNSUPPORTED;
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
  carve(*cfg, h->plan, workspace, &h->P, &h->X, h->kc_store, &h->energy_part, &h->energy_gram, &h->stats_dev);

  StepParams& P = h->P;
  Extra& X = h->X;
  P.dim = cfg->dim;
  P.Mcap = h->plan.Mcap;
  P.Kpad = h->plan.Kpad;
  P.precision = cfg->precision;
  P.c_t = 1.0 / cfg->dt + cfg->alpha * cfg->L;
  P.c_k = cfg->L * cfg->kappa;
  P.L = cfg->L;
  P.a0 = cfg->a0;
  P.tol_als = cfg->tol_als;
  P.tol_enrich = cfg->tol_enrich;
  P.I_max = cfg->I_max;
  P.M_max = cfg->M_max;
  P.fixed_als = cfg->fixed_als_iters;
  P.fixed_modes = cfg->fixed_modes;
  P.seed = cfg->seed;
  const double est = 4.0 * static_cast<double>(N) * cfg->M_max * 2.0 / 1.0e12;
  const double wait_s = cfg->wait_limit_s > 0.0 ? cfg->wait_limit_s : 1.0 + est;
  P.wait_ns = static_cast<unsigned long long>(wait_s * 1e9);
  for (int x = 0; x < cfg->dim; ++x) P.rchunks[x] = h->plan.rchunks[x];

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
    int lead = 2 * s + 1, tail = 2 * s + 1;
    bool uniform = n > lead + tail;
    if (uniform) {
      const double* ref = &h->kband[d][static_cast<size_t>(lead) * w];
      for (int i = lead; i < n - tail && uniform; ++i)
        for (int k = 0; k < w; ++k)
          if (h->kband[d][static_cast<size_t>(i) * w + k] != ref[k]) { uniform = false; break; }
    }
    if (!uniform) { lead = n; tail = 0; }
    std::vector<float2> kc(static_cast<size_t>(lead + tail + 1) * w);
    auto to_df = [](double v) {
      const float hi = static_cast<float>(v);
      return make_float2(hi, static_cast<float>(v - static_cast<double>(hi)));
    };
    for (int i = 0; i < lead; ++i)
      for (int k = 0; k < w; ++k) kc[static_cast<size_t>(i) * w + k] = to_df(h->kband[d][static_cast<size_t>(i) * w + k]);
    for (int t = 0; t < tail; ++t)
      for (int k = 0; k < w; ++k)
        kc[static_cast<size_t>(lead + t) * w + k] = to_df(h->kband[d][static_cast<size_t>(n - tail + t) * w + k]);
    const int srow = uniform ? lead : 0;
    for (int k = 0; k < w; ++k) kc[static_cast<size_t>(lead + tail) * w + k] = to_df(h->kband[d][static_cast<size_t>(srow) * w + k]);
    CTD_CUDA(h, cudaMemcpyAsync(h->kc_store[d], kc.data(), sizeof(float2) * kc.size(), cudaMemcpyHostToDevice,
                                h->stream));
    ctd::KCompressed& k = X.kc[d];
    k.n = n;
    k.b = b;
    k.nlead = lead;
    k.ntail = tail;
    k.rows = h->kc_store[d];
    k.stencil = h->kc_store[d] + static_cast<size_t>(lead + tail) * w;
    k.omega_in = to_df(h->omega[d][n / 2]);
    k.omega_end = to_df(h->omega[d][0]);
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
  while (done < nsteps) {
    const int batch = std::min(nsteps - done, kStatsCap);
    for (int k = 0; k < batch; ++k) {
      h->P.stats = h->stats_dev + k;
      CTD_CUDA(h, cudaMemsetAsync(h->P.barrier, 0, sizeof(unsigned), h->stream));
      CTD_CUDA(h, ctd::launch_step(h->P, h->X, h->grid, h->stream));
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

ctd_status ctd_energy(ctd_handle h, double* energy) {
  if (!h || !energy) return CTD_ERR_ARG;
  if (!h->has_modes) return fail(h, CTD_ERR_STATE, "no field set");
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.status) return fail(h, status_from_bits(st.status), "device status set");
  const int Mk = st.Mk, D = h->cfg.dim;
  CTD_CUDA(h, ctd::launch_convert_modes(h->P, h->X, st.bank, Mk, h->stream));
  int sms = 0;
  CTD_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  const int eg = std::min(1024, 4 * sms);
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

void ctd_destroy(ctd_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
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
  CTD_CUDA(h, ctd::launch_probe_contract(h->P, h->X, h->grid, x, h->stream));
  const int n = h->cfg.n[x], C = h->plan.rchunks[x];
  std::vector<double> part(static_cast<size_t>(n) * C);
  CTD_CUDA(h, cudaMemcpyAsync(part.data(), h->P.rpart, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                              h->stream));
  CTD_CUDA(h, cudaStreamSynchronize(h->stream));
  InstState st;
  ctd_status rs = read_state(h, &st);
  if (rs != CTD_OK) return rs;
  if (st.status) return fail(h, status_from_bits(st.status), "device status set");
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    for (int k = 0; k < C; ++k) r += part[static_cast<size_t>(i) * C + k];
    out[i] = r;
  }
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

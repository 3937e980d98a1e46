/*
 * ctd.h -- C ABI of the GB300 CTD (convolution tensor decomposition) Allen-Cahn solver.
 *
 * The library advances the stabilized semi-implicit Allen-Cahn step (Eq.
 * AC-discrete-semi-stable-K of Lu, Yuan & Guo, arXiv 2410.15519) for a field kept in
 * separated form u = sum_m prod_d u_d^(m) (Eq. CTD).  Each step builds the new field by
 * greedy enrichment; every new mode is computed by the alternating fixed point of Section
 * 3.3 (Eq. ux with K_x, Q_x of Eq. KxQx / Eq. KyQy, derivation in App. D), whose 1D systems
 * use the C-FEM stiffness of Eq. KxxMxx built from the App. B / App. C shape functions.
 * The full-grid nonlinear term M_xy (Eq. KxxMxx) is contracted on the GPU.
 *
 * Conventions for every entry point:
 *  - Every call returns a ctd_status; nothing aborts or exits.  Values > 0 are warnings
 *    (the result is valid), values < 0 are errors (outputs untouched unless stated).
 *  - Device memory: the library allocates none.  The caller queries the workspace size
 *    with ctd_workspace_size, allocates it on the current device and passes it to
 *    ctd_create; the workspace must outlive the handle.  Host memory for the handle itself
 *    is allocated with malloc.
 *  - Caller buffers are never retained after a call returns.
 *  - Work is queued on the CUDA stream given to ctd_create.  Calls that return data to the
 *    host (ctd_energy, ctd_get_modes, ctd_step with stats) synchronise that stream.
 *  - A handle is not thread safe.  Results are deterministic: the same inputs give
 *    bitwise-identical outputs (fixed reduction orders, no floating-point atomics).
 *  - Floating-point arguments are IEEE binary64 unless stated.
 */
#ifndef CTD_H
#define CTD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CTD_OK = 0,
  CTD_STATUS_CAPPED = 1,            /* a step reached M_max modes (Section 3.3 adaptivity cap) */
  CTD_STATUS_ALS_NOT_CONVERGED = 2, /* some mode ended its sweeps without meeting tol_als: at
                                       I_max sweeps, or by the stall rule (als_stall_tol)     */
  CTD_ERR_ARG = -1,                 /* invalid argument or configuration                     */
  CTD_ERR_WORKSPACE = -2,           /* workspace missing, too small or misaligned            */
  CTD_ERR_CUDA = -3,                /* a CUDA runtime call failed                            */
  CTD_ERR_NONFINITE = -4,           /* NaN or Inf met in the modes or a solve                */
  CTD_ERR_TIMEOUT = -5,             /* a grid-wide wait exceeded its time limit              */
  CTD_ERR_STATE = -6,               /* call out of order (e.g. step before initial modes)    */
  CTD_ERR_UNSUPPORTED = -7          /* valid request this build does not implement           */
} ctd_status;

/* Arithmetic of the full-grid nonlinear contraction (all other parts are FP64-accurate).
 * The tensor-core forms rebuild u^k per 128 x 128 tile on tcgen05 tensor cores (FP32
 * accumulation in TMEM), fuse the cubic w(u) into the tile epilogue and sum a tile's columns
 * in FP32, the tiles of a row in FP64.  They differ in how many BF16 terms carry each factor
 * value a (relative error of a reconstructed value, against sum_m |prod_d a_m,d|): */
enum {
  CTD_PREC_FP64 = 0,        /* w(u^k) materialised once per step in FP64, FP64 contraction  */
  CTD_PREC_SPLIT_BF16 = 1,  /* a = hi + lo, 3 products (hi hi, hi lo, lo hi): about 2^-15    */
  CTD_PREC_BF16 = 2,        /* a = hi, one product: about 2^-8                               */
  CTD_PREC_SPLIT3_BF16 = 3  /* a = hi + mid + lo, 6 products (every pair of order <= 2):
                               about 2^-22                                                  */
};

typedef struct {
  int dim;                  /* 2 or 3                                                       */
  int n[3];                 /* nodes per dimension, 4 <= n[d] <= 4096                       */
  double length[3];         /* domain [0, length[d]]                                        */
  int s;                    /* C-FEM patch size, 1..3 (Section 3.2)                         */
  int p;                    /* RBF polynomial order, 1..s (App. B)                          */
  double a;                 /* dilation, natural-coordinate units (App. B)                  */
  double L, kappa, a0, alpha; /* mobility, gradient coefficient, energy coefficient and
                               stabiliser of Eq. AC, Eq. energyfunction, Eq.
                               AC-discrete-semi-stable                                     */
  double dt;                /* time increment                                                */
  int M_max;                /* mode cap per step, 1..128                                    */
  int I_max;                /* fixed-point sweeps per mode, >= 1                            */
  double tol_als;           /* relative Frobenius change of a mode that ends its sweeps     */
  double tol_enrich;        /* a mode with max|prod_d v_d| <= tol_enrich ends the step      */
  int precision;            /* CTD_PREC_*                                                   */
  int fixed_als_iters;      /* > 0: exactly this many sweeps per mode (strict parity)       */
  int fixed_modes;          /* > 0: exactly this many modes per step (strict parity)        */
  unsigned long long seed;  /* SplitMix64 seed for modes without a warm start               */
  double wait_limit_s;      /* limit of each grid-wide wait; <= 0 means 1 second            */
  int grid_ctas;            /* persistent CTAs; <= 0 means one per SM                       */
  double reduced_tol;       /* > 0: reduced integration domain of the nonlinear term
                               (Section 3.3): a block of 128 nodes per dimension (128 x 128
                               in 2D, 128^3 in 3D) drops out of M_xy for the step when
                               max |w(u^k)| over its nodes <= reduced_tol; 0: the whole
                               domain.  Nodal rule only                                      */
  int nonlinear_form;       /* CTD_NONLINEAR_GRID: M_xy as the full nodal integral over the
                               grid (Eq. KxxMxx), tile by tile.  CTD_NONLINEAR_SEPARATED: the
                               separated form of Eq. MxySep, with the exact decomposition of
                               w(u^k) = 4 a0 (u^3 - u) into C(M_k + 2, 3) + M_k separated
                               terms (one per multiset of mode indices, one per mode): every
                               integral becomes a 1D sum, no grid pass.  Requires
                               M_max <= 16 and reduced_tol == 0 (CTD_ERR_ARG otherwise);
                               ctd_step_batch refuses it (CTD_ERR_UNSUPPORTED).            */
  double als_stall_tol;     /* > 0: stall rule of the fixed-point sweeps (Section 3.3's loop
                               until the mode stops changing, read with the paper's absolute
                               example test, the change of the rank-1 term in field units):
                               after at least 3 sweeps a mode whose relative change delta
                               satisfies delta * amp <= als_stall_tol * amp_lead and
                               delta >= delta_prev / 2 ends its sweeps (amp = prod_d max|v_d|,
                               amp_lead that of the step's first mode, the mode's own for the
                               first).  Such a mode has not met tol_als: it is counted in
                               ctd_step_stats.als_stalled and the step returns
                               CTD_STATUS_ALS_NOT_CONVERGED.  0: off (tol_als or I_max only).
                               Same rule for every precision.                              */
  int quad_rule;            /* rule shared by every mass-type integral (M_dd, the nonlinear
                               term M_xy of Eq. KxxMxx, int F in the energy):
                               CTD_QUAD_NODAL: trapezoid weights at the nodes, M_dd =
                               diag(omega) (the default);
                               CTD_QUAD_GAUSS: quad_q Gauss points per element (Section 3.3's
                               Gauss points of each element), M_dd = Phi^T diag(omega_q) Phi,
                               the exact consistent mass for quad_q >= 5, and w(u^k) evaluated
                               at the tensor-product Gauss points and integrated against the
                               shape functions.  Gauss: 1 <= quad_q <= 16, nonlinear_form GRID,
                               reduced_tol 0 and sum over the other dimensions of
                               quad_q (n[d] - 1) <= 12288 for every direction
                               (CTD_ERR_UNSUPPORTED otherwise); ctd_step_batch refuses it.   */
  int quad_q;               /* Gauss points per element (CTD_QUAD_GAUSS)                     */
  int actd_Mc;              /* > 0: adaptive CTD (Section 3.3, "Adaptivity") with critical mode
                               count M_c = actd_Mc: each step runs the greedy loop with the mode
                               budget min(M_max, M_c + 1); a step that commits an (M_c + 1)-th
                               mode discards its separated result and is solved instead on the
                               full tensor-product C-FEM space by fast diagonalisation (the
                               generalised eigenpairs K_d V_d = M_d V_d Lambda_d of every
                               dimension, computed at ctd_create), and the field is then held as
                               the full-grid array of its nodal values; the next step runs CTD
                               from that array (its right-hand side c_t M u^k - int N~ L w(u^k)
                               is one full-grid term, its modes start from the SplitMix64
                               vectors).  0: off.  Requires CTD_PREC_FP64, the nodal rule, the
                               grid nonlinear form and reduced_tol 0 (CTD_ERR_UNSUPPORTED
                               otherwise); ctd_step_batch refuses it.  Uses cuBLAS (FP64 GEMMs
                               of the transforms) and cuSOLVER (the eigenpairs, at create), whose
                               handles allocate their own device memory: the exception to the
                               no-allocation convention above.  ctd_step synchronises after
                               every step to read the switch decision.                        */
  int contraction_form;     /* tensor-core precisions only: how a tile's epilogue forms the
                               weighted sum sum_j c_j w(u_ij) of Eq. KxxMxx (c_j the quadrature
                               weight times the fixed factors of the other dimensions).
                               CTD_CONTRACT_DIRECT: from the reconstructed u, c_j u (u^2 - 1),
                               three FP32 operations per point and c_j read per column.
                               CTD_CONTRACT_CUBE: the column operand is rebuilt every half-sweep
                               with its rows scaled by cbrt(c_j), so that the tensor cores yield
                               v = cbrt(c_j) u and the epilogue sums v^3 = c_j u^3 (two
                               operations per point, no weights); the linear part sum_j c_j u_ij
                               = sum_m a_m,i H_m is added exactly from the Gram products H of the
                               right-hand side.  Exact algebra; its rounding is smaller than the
                               direct form's where |u| is small and larger near |u| = 1, where
                               u^3 and u cancel.
                               CTD_CONTRACT_AUTO (0, the default): the cube form for a step whose
                               field satisfies the bound sum_m prod_d max_i |a_m,d(i)| <= 0.6
                               (then |u^3| <= 0.36 |u| everywhere), else the direct form.  The
                               reduced integration domain and the probes that dump u always use
                               the direct form.  Ignored by CTD_PREC_FP64.                     */
} ctd_config;

enum { CTD_NONLINEAR_GRID = 0, CTD_NONLINEAR_SEPARATED = 1 };
enum { CTD_QUAD_NODAL = 0, CTD_QUAD_GAUSS = 1 };
enum { CTD_CONTRACT_AUTO = 0, CTD_CONTRACT_DIRECT = 1, CTD_CONTRACT_CUBE = 2 };

typedef struct {
  int modes;                /* M of u^{k+1}                                                  */
  int als_sweeps;           /* fixed-point sweeps over all modes tried in the step          */
  int als_sweeps_max;       /* largest per-mode sweep count                                 */
  int capped;               /* 1 if the step ended at M_max                                 */
  int not_converged;        /* 1 if some mode ended without meeting tol_als (I_max or stall) */
  int status;               /* ctd_status of the step                                       */
  int als_stalled;          /* modes whose sweeps the stall rule ended (als_stall_tol)      */
  int als_sweeps_committed; /* sweeps of the committed modes (als_sweeps less those of a mode
                               that the enrichment test discarded)                          */
  int actd_switched;        /* 1 if the step was solved on the full grid (actd_Mc > 0); then
                               modes is the count the greedy loop reached (M_c + 1)          */
  int cube_form;            /* 1 if the step's tensor-core contractions used the cube form
                               (contraction_form), 0 otherwise                               */
} ctd_step_stats;

typedef struct ctd_ctx* ctd_handle;

/* Bytes of device workspace a handle for cfg needs (256-byte aligned base required).
 * Returns CTD_ERR_ARG for an invalid cfg. */
ctd_status ctd_workspace_size(const ctd_config* cfg, size_t* bytes);

/* Create a handle.  Builds the 1D C-FEM stiffness and nodal weights on the host (App. B,
 * App. C, Eq. KxxMxx), uploads them into the workspace (a device pointer owned by the
 * caller, at least ctd_workspace_size bytes) and records cuda_stream (a cudaStream_t, NULL
 * for the legacy default stream).  The current CUDA device must be the workspace's. */
ctd_status ctd_create(const ctd_config* cfg, void* workspace, size_t workspace_bytes,
                      void* cuda_stream, ctd_handle* out);

/* Set u^k to the rank-`rank` separated field whose factor d is the column-major
 * n[d] x rank array modes[d] (mode r at modes[d] + r*n[d]); nodal values, by the
 * Kronecker delta property of the C-FEM shape functions (Section 3.2).  modes[2] is
 * ignored for dim 2.  on_device != 0: the arrays are device pointers.  0 <= rank <= M_max.
 * Copies; resets the step counter to first_step. */
ctd_status ctd_set_initial_modes(ctd_handle h, int rank, const double* const* modes,
                                 int on_device, long long first_step);

/* Advance nsteps time steps (Section 3.3 solution algorithm per step).  Asynchronous on the
 * handle's stream when stats == NULL; otherwise synchronises and writes nsteps records.
 * Returns the most severe status over the steps when stats != NULL. */
ctd_status ctd_step(ctd_handle h, int nsteps, ctd_step_stats* stats);

/* Batched time steps: advance `count` independent instances (handles made by ctd_create on
 * the current device, each with its own configuration, workspace and field) by nsteps time
 * steps each, in one kernel launch per step with one CTA per instance (the many-instance
 * workload of uneven resolution; each instance runs the Section 3.3 step of ctd_step).
 * Work is queued on cuda_stream (a cudaStream_t); the handles' own streams must be idle.
 * workspace: device buffer of ctd_batch_workspace_size(count) bytes, 256-byte aligned, owned
 * by the caller, free again when the call returns with stats != NULL (else once the stream
 * has passed the launches).  stats: NULL, or count * nsteps records, instance-major
 * (stats[i * nsteps + k]); with stats the call synchronises and returns the most severe
 * status.  An instance stepped here is stepped in the same way as by ctd_step: its energy,
 * modes and later ctd_step calls continue from the new state. */
ctd_status ctd_batch_workspace_size(int count, size_t* bytes);
ctd_status ctd_step_batch(const ctd_handle* handles, int count, int nsteps, void* workspace,
                          size_t workspace_bytes, void* cuda_stream, ctd_step_stats* stats);

/* Discrete energy of the current field, E_h = sum_grid omega F(u) + 1/2 kappa u^T K_grad u
 * (energy functional of Section 2.1 with F of Eq. energyfunction; F integrated with the
 * configured rule -- at the nodes, or at the Gauss points with u^k evaluated there -- and
 * the gradient with the exact stiffness and the rule's mass).  FP64.  Synchronises. */
ctd_status ctd_energy(ctd_handle h, double* energy);

/* Copy the current field's factors out: *rank receives M; if M <= capacity, factor d is
 * written column-major into modes_out[d] (n[d] x capacity leading dimension n[d]).
 * Returns CTD_ERR_ARG with *rank set if capacity < M.  A field held on the full grid (after an
 * adaptive-CTD full-grid step) has no factors: CTD_ERR_STATE (read it with ctd_get_field).
 * Synchronises. */
ctd_status ctd_get_modes(ctd_handle h, int capacity, int* rank, double* const* modes_out,
                         int on_device);

/* Full-grid nodal values of the current field (row-major, n[0] x n[1] (x n[2]) doubles, host
 * or device pointer by on_device): rebuilt from the factors, or copied from the full-grid
 * array an adaptive-CTD step left (actd_Mc > 0).  Synchronises. */
ctd_status ctd_get_field(ctd_handle h, double* out, int on_device);

/* Release the handle (not the caller's workspace).  Waits for queued work. */
void ctd_destroy(ctd_handle h);

/* Message of the last failing call on h; for h == NULL, that of the last ctd_create on this
 * thread that failed after validating its arguments (else static text). */
const char* ctd_last_error(ctd_handle h);
const char* ctd_status_string(int status);

/* ---------------------------------------------------------------------------------------
 * Probes: single stages of the step exposed for parity tests and profiling.  Same
 * conventions as above; they run on the handle's stream and synchronise.
 * ------------------------------------------------------------------------------------- */

/* Host-side C-FEM data of dimension d (no GPU work): nodal weights (n[d] values) and the
 * stiffness band (n[d] x (2b+1) row-major, entry (i, j-i+b) = K[i][j], b = 2s+1).
 * Either output may be NULL.  *half_bandwidth receives b. */
ctd_status ctd_probe_cfem(const ctd_config* cfg, int d, double* omega, double* kband,
                          int* half_bandwidth);

/* Host-side operators of the Gauss-point quadrature rule of dimension d (no GPU work; the
 * consistent-mass variant of Eq. KxxMxx, Section 3.3's Gauss points of each element).  q
 * points per element, 1 <= q <= 16, n_q = q (n[d] - 1) points ordered element by element:
 *   x_q[n_q], omega_q[n_q]   points and weights of the composite q-point Gauss-Legendre rule;
 *   phi[n_q][2s+2], phi_col0[n_q]   shape function values, phi[r][k] = N~_{phi_col0[r]+k}(x_r),
 *                            zero past the support of the point's element (nodes e-s .. e+1+s);
 *   mband[n[d]][2b+1]        the mass Phi^T diag(omega) Phi in the layout of ctd_probe_cfem's
 *                            kband (b = 2s+1); for q >= 5 the exact consistent mass;
 *   mass_bounds[2]           bounds lo, hi on the eigenvalues of diag(M)^-1 M (those of a
 *                            Chebyshev solve preconditioned by diag(M)), found by FP64 banded
 *                            Cholesky tests of M - lo diag(M) and hi diag(M) - M and then widened
 *                            by a 1e-6 relative margin; they enclose the spectrum numerically, with
 *                            no proof that the margin covers the tests' rounding errors.
 * Any output may be NULL; the caller owns every buffer.  CTD_ERR_ARG for an invalid
 * configuration, d or q, or a mass that is not positive definite.  A handle created with
 * quad_rule = CTD_QUAD_GAUSS uses the same operators in every step. */
ctd_status ctd_probe_cfem_gauss(const ctd_config* cfg, int d, int q, double* x_q, double* omega_q, double* phi,
                                int* phi_col0, double* mband, double* mass_bounds);

/* Nonlinear contraction of Eq. KxxMxx for direction x with the current field as u^k:
 * nodal rule: out[i] = sum over the other indices of w(u^k) * prod_{d != x} (omega_d v_d),
 * i.e. M_xy u_y / (L omega_x[i]); Gauss rule: out = M_xy u_y / L = Phi_x^T of the weighted
 * sums of w(u^k) at the Gauss points against omega_q (Phi_d v_d) of the other dimensions.
 * v[d] are host arrays of n[d] values (v[x] ignored).  Uses cfg.precision.  The v[d] are copied into the handle's trial factors,
 * which a probe may overwrite (every mode of the next ctd_step starts afresh, so its result
 * is unchanged). */
ctd_status ctd_probe_contract(ctd_handle h, int x, const double* const* v, double* out);

/* Solve (alpha1 diag(omega_x) + alpha2 K_x) y = q with the step's banded solver (FP32
 * Chebyshev semi-iteration on the diag(omega)-scaled operator, or FP32 block cyclic
 * reduction where the Chebyshev row split does not fit, inside iterative refinement with
 * double-float residuals); host arrays of n[x].  Uses the handle's solver vectors and trial
 * factor v[x] as scratch: the next ctd_step starts its modes afresh, so this does not change
 * its result. */
ctd_status ctd_probe_solve(ctd_handle h, int x, double alpha1, double alpha2,
                           const double* q, double* y);

/* Grid values of the current field u^k rebuilt on the tensor cores (handles of a tensor-core
 * precision only): out[i * ncols_pad + c] for the n_pad[x] x ncols_pad tile grid of direction
 * x (rows: nodes of x padded to 128; columns: nodes of the other dimension (2D) or the
 * other dimensions' index pairs (3D, last one padded to 128)), FP32.  scratch: device
 * buffer of at least the output size.  Synchronises.  Sets the handle's trial factors to
 * ones (the next ctd_step starts its modes afresh, so its result is unchanged). */
ctd_status ctd_probe_reconstruct(ctd_handle h, int x, float* out, void* scratch, size_t scratch_bytes);

/* ctd_probe_reconstruct without a caller scratch buffer; the paper has no counterpart (it is
 * a library convenience).  For callers that cannot allocate device memory for the dump: a
 * host program that only holds a handle and has no device allocator of its own, or a run
 * whose device memory is fully committed to the workspace.  The dump goes through a
 * file-scope device array of CTD_RECONSTRUCT_STATIC_BYTES (4 MiB) per device, whose address
 * is looked up once per device on the first call with that device current (do that first
 * call before any stream capture on the device); nothing is allocated by the call itself.
 * Same arguments, layout and result as ctd_probe_reconstruct; the tile grid must fit:
 * n_pad[x] * ncols_pad * 4 bytes <= CTD_RECONSTRUCT_STATIC_BYTES, else CTD_ERR_WORKSPACE
 * (message in ctd_last_error) and nothing is launched.  The current device must be the
 * handle's (CTD_ERR_STATE otherwise).  The used part of the array is zeroed on the handle's
 * stream before the kernel runs.  All handles on one device share the array: calls that
 * overlap in time (other threads or streams on the same device) race and give undefined
 * output; calls from one thread are safe since each call synchronises before returning. */
#define CTD_RECONSTRUCT_STATIC_BYTES ((size_t)4 << 20)
ctd_status ctd_probe_reconstruct_noalloc(ctd_handle h, int x, float* out);

/* Per-phase time of the step kernel, accumulated by CTA 0 from the GPU global timer (each
 * phase includes its closing grid-wide wait).  Copies the seconds accumulated so far into
 * seconds[0 .. nslots) (may be NULL), resets the counters, and turns accumulation on
 * (enable != 0) or off.  Slots: 0 prologue (nonlinear-term preparation), 1 mode start,
 * 2 Gram products + nonlinear contraction, 3 right-hand sides, 4 banded solve,
 * 5 convergence test, 6 mode commit, 7 the cube form's scaled column operand (per
 * half-sweep, contraction_form); inside the banded solve: 8 set-up, 9 first pass,
 * 10 refinement, 11 refinement passes (a count, in units of 1e-9), 14 double-float
 * residuals, 15 inner FP32 solves; 12 Gram products, 13 contraction (timed on the last CTA,
 * whose tile share is a full one; every other slot on CTA 0); tensor-core contraction roles on
 * that last CTA, in SM clock cycles (read as seconds x 1e9): 16 producer waiting for a free
 * stage, 17 MMA issuer waiting for operands, 18 MMA issuer waiting for a free accumulator,
 * 19 MMA issue, 20 epilogue (its first warp) waiting for an accumulator, 21 epilogue work,
 * 22 tiles contracted (a count).  Also counts ctd_probe_solve.  Synchronises. */
ctd_status ctd_probe_trace(ctd_handle h, int enable, double* seconds, int nslots);

#ifdef __cplusplus
}
#endif
#endif /* CTD_H */

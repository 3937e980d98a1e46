"""Python binding of the CTD C ABI (``include/ctd.h``): argument marshalling only.

Every stage of a time step runs in the CUDA library ``libctd.so``; this module allocates the
workspace with PyTorch, passes PyTorch's current CUDA stream, and converts arrays.  There is
no CPU fallback: if the library is missing or cannot be loaded every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctd.so")

PREC_FP64 = 0
PREC_SPLIT_BF16 = 1        # tensor cores, factors as hi + lo BF16 (3 products)
PREC_BF16 = 2              # tensor cores, factors as one BF16 term (1 product)
PREC_SPLIT3_BF16 = 3       # tensor cores, factors as hi + mid + lo BF16 (6 products)
NONLINEAR_GRID = 0         # nonlinear term as the full nodal integral (Eq. KxxMxx)
NONLINEAR_SEPARATED = 1    # separated form (Eq. MxySep) for steps with M_k <= 16
QUAD_NODAL = 0             # mass-type integrals with the nodal rule (M = diag(omega))
QUAD_GAUSS = 1             # Gauss points per element, consistent mass
CONTRACT_AUTO = 0          # tensor-core epilogue: cube form when the field bound allows it
CONTRACT_DIRECT = 1        # tensor-core epilogue: c u (u^2 - 1) from the reconstructed u
CONTRACT_CUBE = 2          # tensor-core epilogue: v^3 with cbrt(c)-scaled columns, exact linear part

STATUS = {0: "CTD_OK", 1: "CTD_STATUS_CAPPED", 2: "CTD_STATUS_ALS_NOT_CONVERGED", -1: "CTD_ERR_ARG",
          -2: "CTD_ERR_WORKSPACE", -3: "CTD_ERR_CUDA", -4: "CTD_ERR_NONFINITE", -5: "CTD_ERR_TIMEOUT",
          -6: "CTD_ERR_STATE", -7: "CTD_ERR_UNSUPPORTED"}


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("length", ctypes.c_double * 3),
                ("s", ctypes.c_int), ("p", ctypes.c_int), ("a", ctypes.c_double),
                ("L", ctypes.c_double), ("kappa", ctypes.c_double), ("a0", ctypes.c_double),
                ("alpha", ctypes.c_double), ("dt", ctypes.c_double), ("M_max", ctypes.c_int),
                ("I_max", ctypes.c_int), ("tol_als", ctypes.c_double), ("tol_enrich", ctypes.c_double),
                ("precision", ctypes.c_int), ("fixed_als_iters", ctypes.c_int),
                ("fixed_modes", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("wait_limit_s", ctypes.c_double), ("grid_ctas", ctypes.c_int),
                ("reduced_tol", ctypes.c_double), ("nonlinear_form", ctypes.c_int),
                ("als_stall_tol", ctypes.c_double), ("quad_rule", ctypes.c_int), ("quad_q", ctypes.c_int),
                ("actd_Mc", ctypes.c_int), ("contraction_form", ctypes.c_int)]


class StepStats(ctypes.Structure):
    _fields_ = [("modes", ctypes.c_int), ("als_sweeps", ctypes.c_int), ("als_sweeps_max", ctypes.c_int),
                ("capped", ctypes.c_int), ("not_converged", ctypes.c_int), ("status", ctypes.c_int),
                ("als_stalled", ctypes.c_int), ("als_sweeps_committed", ctypes.c_int),
                ("actd_switched", ctypes.c_int), ("cube_form", ctypes.c_int)]


class CTDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


def load() -> ctypes.CDLL:
    """Load ``libctd.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_15519_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    pcfg = ctypes.POINTER(Config)
    lib.ctd_workspace_size.argtypes = [pcfg, ctypes.POINTER(sz)]
    lib.ctd_create.argtypes = [pcfg, vp, sz, vp, ctypes.POINTER(vp)]
    lib.ctd_set_initial_modes.argtypes = [vp, i, ctypes.POINTER(vp), i, ctypes.c_longlong]
    lib.ctd_step.argtypes = [vp, i, ctypes.POINTER(StepStats)]
    lib.ctd_energy.argtypes = [vp, ctypes.POINTER(d)]
    lib.ctd_get_modes.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(vp), i]
    lib.ctd_get_field.argtypes = [vp, vp, i]
    lib.ctd_destroy.argtypes = [vp]
    lib.ctd_destroy.restype = None
    lib.ctd_last_error.argtypes = [vp]
    lib.ctd_last_error.restype = ctypes.c_char_p
    lib.ctd_status_string.argtypes = [i]
    lib.ctd_status_string.restype = ctypes.c_char_p
    lib.ctd_probe_cfem.argtypes = [pcfg, i, vp, vp, ctypes.POINTER(i)]
    lib.ctd_probe_cfem_gauss.argtypes = [pcfg, i, i, vp, vp, vp, vp, vp, vp]
    lib.ctd_probe_contract.argtypes = [vp, i, ctypes.POINTER(vp), vp]
    lib.ctd_probe_solve.argtypes = [vp, i, d, d, vp, vp]
    lib.ctd_probe_trace.argtypes = [vp, i, vp, i]
    lib.ctd_probe_reconstruct.argtypes = [vp, i, vp, vp, sz]
    lib.ctd_probe_reconstruct_noalloc.argtypes = [vp, i, vp]
    lib.ctd_batch_workspace_size.argtypes = [i, ctypes.POINTER(sz)]
    lib.ctd_step_batch.argtypes = [ctypes.POINTER(vp), i, i, vp, sz, vp, ctypes.POINTER(StepStats)]
    for f in ("ctd_workspace_size", "ctd_create", "ctd_set_initial_modes", "ctd_step", "ctd_energy",
              "ctd_get_modes", "ctd_get_field", "ctd_probe_cfem", "ctd_probe_contract", "ctd_probe_solve", "ctd_probe_trace",
              "ctd_probe_reconstruct", "ctd_probe_reconstruct_noalloc", "ctd_batch_workspace_size",
              "ctd_step_batch"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def make_config(dim, n, length, s, p, a, L, kappa, a0, alpha, dt, M_max, I_max, tol_als, tol_enrich,
                precision=PREC_FP64, fixed_als_iters=0, fixed_modes=0, seed=0, wait_limit_s=0.0,
                grid_ctas=0, reduced_tol=0.0, nonlinear_form=0, als_stall_tol=0.0, quad_rule=0,
                quad_q=0, actd_Mc=0, contraction_form=CONTRACT_AUTO) -> Config:
    c = Config()
    c.dim = dim
    for k in range(3):
        c.n[k] = int(n[k]) if k < dim else 0
        c.length[k] = float(length[k]) if k < dim else 0.0
    c.s, c.p, c.a = int(s), int(p), float(a)
    c.L, c.kappa, c.a0, c.alpha, c.dt = float(L), float(kappa), float(a0), float(alpha), float(dt)
    c.M_max, c.I_max = int(M_max), int(I_max)
    c.tol_als, c.tol_enrich = float(tol_als), float(tol_enrich)
    c.precision, c.fixed_als_iters, c.fixed_modes = int(precision), int(fixed_als_iters), int(fixed_modes)
    c.seed, c.wait_limit_s, c.grid_ctas = int(seed), float(wait_limit_s), int(grid_ctas)
    c.reduced_tol = float(reduced_tol)
    c.nonlinear_form = int(nonlinear_form)
    c.als_stall_tol = float(als_stall_tol)
    c.quad_rule, c.quad_q = int(quad_rule), int(quad_q)
    c.actd_Mc = int(actd_Mc)
    c.contraction_form = int(contraction_form)
    return c


def config_from_workload(w, precision=PREC_FP64, **overrides) -> Config:
    """Config of a ``workloads.Workload`` (paper symbols L, kappa, a0, alpha)."""
    args = dict(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                tol_enrich=w.tol_enrich, precision=precision, seed=w.seed)
    args.update(overrides)
    return make_config(**args)


def _check(lib, h, st, what):
    if st < 0:
        msg = lib.ctd_last_error(h).decode() if h else lib.ctd_status_string(st).decode()
        if not h:
            last = lib.ctd_last_error(None).decode()
            if last != "no handle":
                msg += f" ({last})"
        raise CTDError(st, f"{what}: {msg}")
    return st


def workspace_size(cfg: Config) -> int:
    lib = load()
    n = ctypes.c_size_t(0)
    _check(lib, None, lib.ctd_workspace_size(ctypes.byref(cfg), ctypes.byref(n)), "ctd_workspace_size")
    return n.value


def probe_cfem(cfg: Config, d: int):
    """Host-side C-FEM data of dimension d: (omega, band [n x (2b+1)], b)."""
    lib = load()
    b = ctypes.c_int(0)
    _check(lib, None, lib.ctd_probe_cfem(ctypes.byref(cfg), d, None, None, ctypes.byref(b)), "probe_cfem")
    n = cfg.n[d]
    om = np.zeros(n)
    kb = np.zeros((n, 2 * b.value + 1))
    _check(lib, None, lib.ctd_probe_cfem(ctypes.byref(cfg), d, om.ctypes.data, kb.ctypes.data, ctypes.byref(b)),
           "probe_cfem")
    return om, kb, b.value


def probe_cfem_gauss(cfg: Config, d: int, q: int, bounds: bool = True):
    """Host-side Gauss-rule operators of dimension d: (x_q, omega_q, Phi as a dense n_q x n
    array, mass band [n x (2b+1)], (lo, hi) bounds of the spectrum of diag(M)^-1 M, or None
    when ``bounds`` is False)."""
    lib = load()
    n, s = cfg.n[d], cfg.s
    nq, wphi, w = q * (n - 1), 2 * s + 2, 2 * (2 * s + 1) + 1
    xq, om = np.zeros(nq), np.zeros(nq)
    phi = np.zeros((nq, wphi))
    col0 = np.zeros(nq, dtype=np.int32)
    mb = np.zeros((n, w))
    bd = np.zeros(2)
    _check(lib, None, lib.ctd_probe_cfem_gauss(ctypes.byref(cfg), d, q, xq.ctypes.data, om.ctypes.data,
                                               phi.ctypes.data, col0.ctypes.data, mb.ctypes.data,
                                               bd.ctypes.data if bounds else None),
           "probe_cfem_gauss")
    dense = np.zeros((nq, n))
    for r in range(nq):
        k = min(wphi, n - int(col0[r]))
        dense[r, col0[r]:col0[r] + k] = phi[r, :k]
    return xq, om, dense, mb, ((float(bd[0]), float(bd[1])) if bounds else None)


_batch_keep: List = []


def step_batch(solvers: Sequence["Solver"], nsteps: int = 1, stats: bool = True, stream=None, sync: bool = True):
    """Advance independent instances together, one CTA per instance per launch
    (ctd_step_batch).  Returns per-instance lists of step records when stats is true; without
    stats and with sync false the launches are left queued on the stream."""
    import torch
    lib = load()
    count = len(solvers)
    nb = ctypes.c_size_t(0)
    _check(lib, None, lib.ctd_batch_workspace_size(count, ctypes.byref(nb)), "ctd_batch_workspace_size")
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    handles = (ctypes.c_void_p * count)(*[s.h for s in solvers])
    stream = stream if stream is not None else torch.cuda.current_stream()
    for s in solvers:
        s.stream.synchronize()
    rec = (StepStats * (count * nsteps))() if stats else None
    st = lib.ctd_step_batch(handles, count, nsteps, ctypes.c_void_p(ws.data_ptr()), nb.value,
                            ctypes.c_void_p(stream.cuda_stream), rec)
    if st < 0:
        bad = next((s.h for s in solvers if lib.ctd_last_error(s.h)), None)
        _check(lib, bad, st, "ctd_step_batch")
    if not stats:
        if sync:
            stream.synchronize()
        else:
            _batch_keep.append(ws)   # the queued launches still read it
            del _batch_keep[:-4]
        return None
    out = []
    for i in range(count):
        out.append([dict(modes=r.modes, als_sweeps=r.als_sweeps, als_sweeps_max=r.als_sweeps_max,
                         capped=bool(r.capped), not_converged=bool(r.not_converged), status=r.status,
                         als_stalled=r.als_stalled,
                         als_sweeps_committed=r.als_sweeps_committed,
                         actd_switched=bool(r.actd_switched), cube_form=bool(r.cube_form))
                    for r in rec[i * nsteps:(i + 1) * nsteps]])
    return out


class Solver:
    """One CTD Allen-Cahn instance on the current CUDA device."""

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.lib = load()
        self.cfg = cfg
        self.torch = torch
        nbytes = workspace_size(cfg)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        st = self.lib.ctd_create(ctypes.byref(cfg), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(self.lib, None, st, "ctd_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.ctd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_initial_modes(self, modes: Sequence, first_step: int = 0):
        """modes[d]: n_d x rank array (numpy on the host, or a CUDA torch tensor)."""
        torch = self.torch
        rank = int(modes[0].shape[1])
        on_dev = isinstance(modes[0], torch.Tensor) and modes[0].is_cuda
        keep = []
        ptrs = (ctypes.c_void_p * 3)()
        for d in range(self.cfg.dim):
            if on_dev:
                t = modes[d].to(torch.float64).t().contiguous()      # column-major n x rank
                keep.append(t)
                ptrs[d] = t.data_ptr()
            else:
                a = np.asfortranarray(np.asarray(modes[d], dtype=np.float64))
                keep.append(a)
                ptrs[d] = a.ctypes.data
        st = self.lib.ctd_set_initial_modes(self.h, rank, ptrs, 1 if on_dev else 0, int(first_step))
        if on_dev:
            self.stream.synchronize()
        _check(self.lib, self.h, st, "ctd_set_initial_modes")

    def step(self, nsteps: int = 1, stats: bool = True):
        if not stats:
            _check(self.lib, self.h, self.lib.ctd_step(self.h, nsteps, None), "ctd_step")
            return None
        rec = (StepStats * nsteps)()
        st = self.lib.ctd_step(self.h, nsteps, rec)
        _check(self.lib, self.h, st, "ctd_step")
        return [dict(modes=r.modes, als_sweeps=r.als_sweeps, als_sweeps_max=r.als_sweeps_max,
                     capped=bool(r.capped), not_converged=bool(r.not_converged), status=r.status,
                         als_stalled=r.als_stalled,
                         als_sweeps_committed=r.als_sweeps_committed,
                         actd_switched=bool(r.actd_switched), cube_form=bool(r.cube_form)) for r in rec]

    def energy(self) -> float:
        e = ctypes.c_double(0.0)
        _check(self.lib, self.h, self.lib.ctd_energy(self.h, ctypes.byref(e)), "ctd_energy")
        return e.value

    def get_modes(self, device: bool = False) -> List:
        torch = self.torch
        r = ctypes.c_int(0)
        st = self.lib.ctd_get_modes(self.h, 0, ctypes.byref(r), None, 0)
        if st < 0 and r.value == 0:
            _check(self.lib, self.h, st, "ctd_get_modes")
        rank = r.value
        ptrs = (ctypes.c_void_p * 3)()
        outs = []
        for d in range(self.cfg.dim):
            if device:
                t = torch.empty((rank, self.cfg.n[d]), dtype=torch.float64, device="cuda")
                ptrs[d] = t.data_ptr()
            else:
                t = np.zeros((self.cfg.n[d], rank), order="F")
                ptrs[d] = t.ctypes.data
            outs.append(t)
        if rank:
            _check(self.lib, self.h, self.lib.ctd_get_modes(self.h, rank, ctypes.byref(r), ptrs, 1 if device else 0),
                   "ctd_get_modes")
        if device:
            return [t.t() for t in outs]
        return [np.ascontiguousarray(t) for t in outs]

    def get_field(self) -> np.ndarray:
        """Full-grid nodal values of the current field (host array, n[0] x n[1] (x n[2]))."""
        shape = tuple(self.cfg.n[d] for d in range(self.cfg.dim))
        out = np.zeros(shape)
        _check(self.lib, self.h, self.lib.ctd_get_field(self.h, out.ctypes.data, 0), "ctd_get_field")
        return out

    def probe_contract(self, x: int, v: Sequence[np.ndarray]) -> np.ndarray:
        ptrs = (ctypes.c_void_p * 3)()
        keep = []
        for d in range(self.cfg.dim):
            a = np.ascontiguousarray(np.asarray(v[d], dtype=np.float64))
            keep.append(a)
            ptrs[d] = a.ctypes.data
        out = np.zeros(self.cfg.n[x])
        _check(self.lib, self.h, self.lib.ctd_probe_contract(self.h, x, ptrs, out.ctypes.data), "probe_contract")
        return out

    def probe_reconstruct(self, x: int, rows_pad: int, cols_pad: int) -> np.ndarray:
        """u^k on the tile grid of direction x rebuilt on the tensor cores (FP32)."""
        torch = self.torch
        out = np.zeros((rows_pad, cols_pad), dtype=np.float32)
        scratch = torch.empty(out.nbytes, dtype=torch.uint8, device="cuda")
        _check(self.lib, self.h, self.lib.ctd_probe_reconstruct(self.h, x, out.ctypes.data,
                                                                ctypes.c_void_p(scratch.data_ptr()), out.nbytes),
               "probe_reconstruct")
        return out

    def probe_reconstruct_noalloc(self, x: int, rows_pad: int, cols_pad: int) -> np.ndarray:
        """probe_reconstruct through the library's static dump array (no scratch allocated)."""
        out = np.zeros((rows_pad, cols_pad), dtype=np.float32)
        _check(self.lib, self.h, self.lib.ctd_probe_reconstruct_noalloc(self.h, x, out.ctypes.data),
               "probe_reconstruct_noalloc")
        return out

    TRACE_PHASES = ("prologue", "mode_start", "gram_contract", "rhs", "solve", "converge", "commit", "scale_operand")

    def trace(self, enable: bool = True) -> dict:
        """Seconds per step-kernel phase accumulated since the last call; (re)starts or stops
        accumulation."""
        out = np.zeros(24)
        _check(self.lib, self.h, self.lib.ctd_probe_trace(self.h, 1 if enable else 0, out.ctypes.data, 24),
               "probe_trace")
        d = dict(zip(self.TRACE_PHASES, out[:len(self.TRACE_PHASES)].tolist()))
        d.update(solve_factor=out[8], solve_first=out[9], solve_refine=out[10], solve_passes=out[11] * 1e9,
                 gram=out[12], contract=out[13], solve_residual=out[14], solve_inner=out[15])
        # tensor-core contraction roles on the traced CTA, in SM clock cycles
        for k, name in enumerate(("tc_producer_wait", "tc_mma_wait_operands", "tc_mma_wait_accumulator",
                                  "tc_mma_issue", "tc_epilogue_wait", "tc_epilogue_work", "tc_tiles")):
            d[name + ("" if name == "tc_tiles" else "_cycles")] = out[16 + k] * 1e9
        return d

    def probe_solve(self, x: int, alpha1: float, alpha2: float, q: np.ndarray) -> np.ndarray:
        q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        y = np.zeros(self.cfg.n[x])
        _check(self.lib, self.h, self.lib.ctd_probe_solve(self.h, x, float(alpha1), float(alpha2), q.ctypes.data,
                                                          y.ctypes.data), "probe_solve")
        return y

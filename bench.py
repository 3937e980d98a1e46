"""Benchmark: CTD Allen-Cahn time steps/s on one GB300 (and equivalent DOF-updates/s).

Headline workload (default ``--workload c3``): 3D, 1024^3 nodes (1.07G equivalent grid
points, never materialised), C-FEM s = p = 3, eps = 0.01, S = 2, dt = 2e-3, up to 80 modes,
seeded rank-10 cosine initial condition.  One "step" is one full time step of the CTD solver
(greedy enrichment with fixed-point sweeps and the full-grid nonlinear contraction), one
kernel launch through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3|c2|c1|c4]
                  [--precision mixed|fp64] [--stall TOL] [--extras c1,c2,c4|none]
                  [--impl ours|reference]

The headline is the mixed form (split-BF16 tensor-core contraction, FP64-accurate solves,
Gram products and energy).  Both arithmetics run under the same stop rules: the relative
change tol_als = 1e-8 per mode, the sweep cap I_max = 50 and the stall rule
``als_stall_tol`` (``--stall``, 1e-6 by default: a mode whose change in units of the
step's leading mode is below it and no longer shrinking ends its sweeps, counted as
stalled).  The plain FP64 form is timed beside it under the same rules, and both again with
the stall rule off.  The error of the mixed form is measured against the FP64 form on the
GPU (the oracle cannot hold the 3D grids).  Prints one JSON line.  Under torchrun (N > 1)
every rank advances its own replica (weak scaling, no collective on the data path); rank 0
prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "CTD time steps/s and equivalent grid DOF-updates/s at fixed error vs FP64 oracle"
UNIT = "time_steps/s"
STALL_DEFAULT = 1e-6
SMS = 152
# Per single-instance workload: steps of the FP64-vs-mixed accuracy run and of the side legs
# (plain FP64 form, stall rule off), and the oracle's sample grid when the workload's own grid
# is too large for it (None: the workload itself).
PLAN = {"c0": dict(err_steps=10, side_steps=10, oracle_n=None),
        "c1": dict(err_steps=10, side_steps=10, oracle_n=None),
        "c1i": dict(err_steps=5, side_steps=5, oracle_n=None),
        "c2": dict(err_steps=2, side_steps=3, oracle_n=128),
        "c3": dict(err_steps=2, side_steps=2, oracle_n=128)}
FP64_NOMINAL_TFLOPS = 1.25   # nominal FP64 (non-tensor) rate of the part, from the pool's table
PRODUCTS = {"mixed": 3, "bf16": 1, "split3": 6}   # BF16 products per mode and grid point


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def alu_peak_tops(pk) -> float:
    """FP32 lane operations per second of the whole GPU: 152 SMs x 128 FP32 lanes x the
    maximum SM clock."""
    return SMS * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


# --------------------------------------------------------------------------- CPU oracle leg
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np, workloads
from oracle import ctd
over = {over!r}
w = workloads.preset({name!r}, **over)
prob = ctd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                   a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                   tol_enrich=w.tol_enrich, seed=w.seed, als_stall_tol={stall!r})
t0 = time.perf_counter(); ops = ctd.build_operators(prob); t_setup = time.perf_counter() - t0
A = workloads.initial_modes(w)
steps, times, stats = 0, [], []
budget = {budget}
t_all = time.perf_counter()
while steps < {max_steps} and (steps == 0 or time.perf_counter() - t_all < budget):
    t0 = time.perf_counter()
    A, st = ctd.step(prob, ops, A, steps)
    times.append(time.perf_counter() - t0)
    stats.append(dict(modes=st["modes"], sweeps=sum(st["als_iters"])))
    steps += 1
    if steps == 1 and {save!r}:
        np.savez({out!r} + ".npz", *A)
json.dump(dict(steps=steps, times=times, setup_s=t_setup, stats=stats, n=list(w.n)), open({out!r}, "w"))
"""


def run_oracle(name: str, max_steps: int, budget_s: float, stall: float, sample_n=None, save=True):
    """Time the oracle as it stands on the host, single-threaded BLAS, in a fresh process: on
    the workload itself, or on its parameters with `sample_n` nodes per dimension."""
    fd, out = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    w = workloads.preset(name)
    over = {} if sample_n is None else dict(n=tuple([sample_n] * w.dim))
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, over=over, stall=stall, budget=budget_s,
                                 max_steps=max_steps, out=out, save=save and sample_n is None)
    subprocess.run([sys.executable, "-c", code], check=True, env=env)
    res = json.load(open(out))
    modes = None
    if os.path.exists(out + ".npz"):
        z = np.load(out + ".npz")
        modes = [z[k] for k in sorted(z.files, key=lambda s: int(s.split("_")[1]))]
        os.remove(out + ".npz")
    os.remove(out)
    return res, modes


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_baseline(name: str, stall: float, budget_s: float, max_steps: int = 1, save=True):
    """The oracle's time steps/s on the workload: its own grid where the oracle holds it, else
    a sample of the same parameters on a 128^D grid scaled by grid points (the oracle's step is
    dominated by its full-grid contractions, linear in the grid points; the sample's arrays fit
    the host caches, so the scaled figure favours the CPU)."""
    w = workloads.preset(name)
    sn = PLAN.get(name, {}).get("oracle_n")
    res, modes = run_oracle(name, max_steps, budget_s, stall, sample_n=sn, save=save)
    t_step = sum(res["times"]) / res["steps"]
    n_s = int(np.prod(res["n"]))
    value = (1.0 / t_step) * (n_s / w.grid_points)
    if sn is None:
        sample = f"first {res['steps']} time step(s) of {name} from the initial condition"
    else:
        sample = (f"first {res['steps']} time step(s) of the {name} parameters on a {sn}^{w.dim} grid "
                  f"({n_s} points, {res['stats'][0]['modes']} modes, {res['stats'][0]['sweeps']} sweeps, "
                  f"{t_step:.2f} s/step), scaled by grid points to {w.grid_points}")
    info = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": sample + f"; single-threaded BLAS, stall rule {stall:g}",
            "nproc": os.cpu_count(), "cpu_model": cpu_model(), "oracle_s_per_step": t_step}
    return info, modes, res


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swpc=parts[8]))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("swpc", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- ranks
def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """Slowest rank's value (replicas run independently; the job ends with the last one)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_units(steps: int, world: int) -> int:
    """Time steps advanced by the whole job: every rank advances its own instance."""
    return steps * world


# --------------------------------------------------------------------------- rooflines
def epilogue_ops(cube: bool) -> float:
    """FP32 operations per grid point of the contraction epilogue: the direct form's
    u*u - 1, times (u c_j), into the row sum (3); the cube form's v*v, times v into the row
    sum (2)."""
    return 2.0 if cube else 3.0


def half_sweep_roof_s(w, precision: str, Mk: int, pk: dict, cube: bool = False) -> dict:
    """Roofline time of one half-sweep's nonlinear contraction over the whole grid (the only
    term of the step that grows with the grid): the largest of
      tensor: 2 K_eff N flops at the BF16 burst peak (K_eff = 3 Mk for the split product),
      alu:    the epilogue's FP32 operations per grid point (3 direct, 2 cube form) on
              152 x 128 FP32 lanes at the maximum SM clock,
      hbm:    the operands' bytes (factor rows, K_eff BF16 values each) at the copy bandwidth;
    FP64 path: one FP64 multiply-add per grid point on the FP64 pipe, or the 8 N bytes of the
    materialised w(u^k) grid from HBM, whichever is slower."""
    N = float(w.grid_points)
    if precision == "fp64":
        t_f = 2.0 * N / (FP64_NOMINAL_TFLOPS * 1e12)
        t_b = 8.0 * N / (pk["hbm_gbs"] * 1e9)
        return {"fp64": t_f, "hbm": t_b}
    keff = PRODUCTS[precision] * Mk
    t_tensor = 2.0 * keff * N / (pk["bf16_tflops"] * 1e12)
    t_alu = epilogue_ops(cube) * N / (alu_peak_tops(pk) * 1e12)
    t_hbm = 2.0 * keff * sum(w.n) / (pk["hbm_gbs"] * 1e9)
    return {"tensor": t_tensor, "alu": t_alu, "hbm": t_hbm}


def step_roofline(w, precision, ranks_in, stats, times_ms, pk, pk_kind, traffic):
    """Roofline of the step kernel over the timed steps: the sum over steps of (half-sweeps x
    the half-sweep roof at that step's M_k) against the measured launch times.  achieved and
    peak are in the unit of the bound that dominates."""
    roof = {}
    for mk, st in zip(ranks_in, stats):
        hs = st["als_sweeps"] * w.dim
        for k, v in half_sweep_roof_s(w, precision, mk, pk, st.get("cube_form", False)).items():
            roof[k] = roof.get(k, 0.0) + hs * v
    t = sum(times_ms) / 1e3
    bound = max(roof, key=roof.get)
    N = float(w.grid_points)
    hs_all = sum(st["als_sweeps"] for st in stats) * w.dim
    if bound == "alu":
        ops = sum(epilogue_ops(st.get("cube_form", False)) * st["als_sweeps"] * w.dim for st in stats)
        achieved, peak, unit = ops * N / t / 1e12, alu_peak_tops(pk), "TFLOP/s"
        peak_kind = ("FP32 lane operations (per grid point and half-sweep: 3 in the direct form, 2 in the cube "
                     f"form), peak = 152 SMs x 128 lanes x {pk.get('sm_max_mhz', 2070.0):.0f} MHz, derived from "
                     "unit counts and the maximum clock")
    elif bound == "tensor":
        flops = sum(2.0 * PRODUCTS[precision] * mk * N * st["als_sweeps"] * w.dim for mk, st in zip(ranks_in, stats))
        achieved, peak, unit = flops / t / 1e12, pk["bf16_tflops"], "TFLOP/s"
        peak_kind = f"bf16 dense burst, {pk_kind} (of {pk_kind})"
    elif bound == "fp64":
        achieved, peak, unit = 2.0 * N * hs_all / t / 1e12, FP64_NOMINAL_TFLOPS, "TFLOP/s"
        peak_kind = "nominal FP64 rate of the part (the pool's table); a throughput probe measured 1.0"
    else:
        byts = 8.0 * N * hs_all if precision == "fp64" else 0.0
        achieved, peak, unit = byts / t / 1e9, pk["hbm_gbs"], "GB/s"
        peak_kind = f"copy bandwidth, {pk_kind} (of {pk_kind})"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": roof[bound] / t,
            "traffic": traffic, "peak_kind": peak_kind, "roof_s_per_step": {k: v / len(stats) for k, v in roof.items()},
            "kernel": "ctd::step_kernel (whole persistent time step, one launch per step)",
            "note": "frac = sum over the timed steps of half-sweeps x the contraction's roofline time at that "
                    "step's M_k (max of tensor, FP32 epilogue, operand bytes) / measured launch time; the "
                    "1D solves, Gram products and grid-wide waits have no roofline term"}


def last_cta_tile_share(w, G: int = SMS) -> float:
    """Fraction of direction 0's 128 x 128 tiles that the last of G CTAs contracts (the
    library's split: the first 16 CTAs, which also form the Gram partial sums, weigh 1, the
    others 8; CTA c starts at floor(T cum(c) / cum(G)))."""
    T = 1
    for d in range(w.dim):
        T *= -(-w.n[d] // 128)
    L = min(G, 16)
    cum = lambda c: c if c <= L else L + 8 * (c - L)
    lo = T * cum(G - 1) // cum(G)
    return (T - lo) / T


def contraction_roof_us(w, Mk: float, pk: dict, precision: str = "mixed", cube: bool = False) -> dict:
    """Roofline time of the last CTA's share of one half-sweep's tensor-core contraction (the
    phase is timed on that CTA): the larger of the split reconstruction on the tensor cores
    (2 * 3Mk flops per grid point at one SM's share of the BF16 burst peak) and the fused
    epilogue on the FP32 pipes (3 or 2 operations per grid point on 128 lanes at the maximum
    clock)."""
    n_cta = float(w.grid_points) * last_cta_tile_share(w)
    t_tensor = 2.0 * PRODUCTS[precision] * Mk * n_cta / (pk["bf16_tflops"] * 1e12 / SMS)
    t_alu = epilogue_ops(cube) * n_cta / (128 * pk.get("sm_max_mhz", 2070.0) * 1e6)
    bound = "tensor" if t_tensor >= t_alu else "alu"
    return {"roof_us": 1e6 * max(t_tensor, t_alu), "bound": bound, "tensor_us": 1e6 * t_tensor, "alu_us": 1e6 * t_alu,
            "grid_points": n_cta}


DEVICE_SOURCES = ("ctd_common.cuh", "ctd_contract_tc.cuh", "ctd_kernels.cu", "ctd_kernels_sep.cu", "ctd_solve.cuh",
                  "ctd_step.cuh")


def source_hash() -> str:
    """Digest of the device-code sources (ties stored ncu counters to the kernels they measured)."""
    h = hashlib.sha256()
    for f in DEVICE_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(ROOT, "paper_2410_15519_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(key: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was taken on
    the current device sources (else None)."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    except (OSError, ValueError):
        return None
    e = rec.get(key)
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- GPU legs
PRECISIONS = ("fp64", "mixed", "bf16", "split3")


def prec_code(ctd, precision):
    """fp64: FP64 contraction; mixed: split-BF16 (hi + lo) tensor cores; bf16: one BF16 term;
    split3: hi + mid + lo."""
    return {"fp64": ctd.PREC_FP64, "mixed": ctd.PREC_SPLIT_BF16, "bf16": ctd.PREC_BF16,
            "split3": ctd.PREC_SPLIT3_BF16}[precision]


def timed_run(ctd, torch, w, precision, steps, warmup, flush, clocks=None, over=None):
    """Advance `steps` time steps after `warmup`; one step kernel launch each, bracketed by CUDA
    events on the solver's stream, L2 flushed between steps."""
    solver = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, precision), **(over or {})))
    stream = solver.stream
    solver.set_initial_modes(workloads.initial_modes(w))
    for _ in range(warmup):
        solver.step(1, stats=False)
    torch.cuda.synchronize()
    rank0 = solver.get_modes()[0].shape[1]
    if clocks:
        clocks.start()
    times_ms, stats = [], []
    torch.cuda.synchronize()
    for _ in range(steps):
        flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = solver.step(1)[0]
        ev1.record(stream)
        ev1.synchronize()
        times_ms.append(ev0.elapsed_time(ev1))
        stats.append(st)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    return solver, times_ms, stats, rank0, clk


def field_rel_l2(A, B):
    """Relative nodal L2 distance ||u_A - u_B|| / ||u_B|| of two separated fields, rebuilt in
    FP64 on the GPU slab by slab (a Gram-matrix form would cancel catastrophically at the
    differences measured here)."""
    import torch
    ta = [torch.as_tensor(a, dtype=torch.float64, device="cuda") for a in A]
    tb = [torch.as_tensor(b, dtype=torch.float64, device="cuda") for b in B]
    n0 = ta[0].shape[0]
    num = den = 0.0
    step = 64 if len(ta) == 3 else n0
    for i0 in range(0, n0, step):
        i1 = min(n0, i0 + step)
        if len(ta) == 2:
            ua, ub = ta[0][i0:i1] @ ta[1].T, tb[0][i0:i1] @ tb[1].T
        else:
            ua = torch.einsum("im,jm,km->ijk", ta[0][i0:i1], ta[1], ta[2])
            ub = torch.einsum("im,jm,km->ijk", tb[0][i0:i1], tb[1], tb[2])
        num += float(torch.sum((ua - ub) ** 2))
        den += float(torch.sum(ub ** 2))
    return (num / den) ** 0.5 if den > 0 else num ** 0.5


def leg_summary(times_ms, stats, w):
    ms = sum(times_ms) / len(times_ms)
    hs = sum(s["als_sweeps"] for s in stats) * w.dim
    return {"steps": len(times_ms), "ms_per_step": ms, "value": 1e3 / ms, "unit": UNIT,
            "als_sweeps_per_step": [s["als_sweeps"] for s in stats],
            "als_stalled_per_step": [s["als_stalled"] for s in stats],
            "us_per_half_sweep": 1e3 * sum(times_ms) / max(1, hs)}


def run_single(ctd, torch, w, args, flush, local_rank, headline=True):
    """All measurements of one single-instance workload (module docstring)."""
    stall = args.stall
    plan = PLAN.get(w.name, dict(err_steps=2, side_steps=2, oracle_n=128))
    over = dict(als_stall_tol=stall)
    steps = args.steps if headline else args.extra_steps
    clocks = ClockSampler(local_rank) if headline else None
    solver, times_ms, stats, rank0, clk = timed_run(ctd, torch, w, args.precision, steps, args.warmup, flush,
                                                     clocks, over)
    ranks_in = [rank0] + [st["modes"] for st in stats[:-1]]
    out = dict(times_ms=times_ms, stats=stats, clocks=clk, ranks_in=ranks_in, mk_mean=sum(ranks_in) / len(ranks_in))
    # per-phase device time of two more steps (global-timer trace of CTA 0 / the last CTA)
    solver.trace(True)
    st_tr = solver.step(2)
    tr = solver.trace(False)
    hs = sum(s["als_sweeps"] for s in st_tr) * w.dim
    out["phase_us_per_half_sweep"] = {k: 1e6 * v / max(1, hs) for k, v in tr.items()
                                      if k in ("gram_contract", "gram", "contract", "rhs", "solve", "converge")}
    if tr.get("tc_tiles", 0) > 0:
        # the tensor-core contraction's roles on the traced (last) CTA, SM cycles per tile
        out["contraction_role_cycles_per_tile"] = {
            k[3:-7]: v / tr["tc_tiles"] for k, v in tr.items() if k.startswith("tc_") and k.endswith("_cycles")}
    solver.close()
    if headline:
        # End to end through the C ABI with host buffers, on the same steps as the first timed
        # ones (a fresh solver from the initial condition, the same warm-up): every step the H2D
        # copy of u^k's factors, the step, the D2H read of u^{k+1}'s factors.
        n_e2e = min(steps, args.e2e_steps)
        solver = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, args.precision), **over))
        solver.set_initial_modes(workloads.initial_modes(w))
        solver.step(args.warmup, stats=False)
        modes_host = solver.get_modes()
        bi = bo = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            bi += sum(m.nbytes for m in modes_host)
            solver.set_initial_modes(modes_host, first_step=args.warmup + k)
            solver.step(1)
            modes_host = solver.get_modes()
            bo += sum(m.nbytes for m in modes_host)
        torch.cuda.synchronize()
        out["e2e"] = dict(steps=n_e2e, seconds=time.perf_counter() - t0, h2d=bi / max(1, n_e2e),
                          d2h=bo / max(1, n_e2e),
                          device_ms_same_steps=sum(times_ms[:n_e2e]))
        solver.close()
    if getattr(args, "quick", False):
        out["accuracy"], out["first_step_modes"], out["side"], out["ladder"] = {}, {}, {}, {}
        return out
    # accuracy: both arithmetics from the initial condition under the same rules
    traj = {}
    for prec in ("mixed", "fp64"):
        sv = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, prec), **over))
        sv.set_initial_modes(workloads.initial_modes(w))
        energies, first, sst = [sv.energy()], None, []
        for k in range(plan["err_steps"]):
            sst.append(sv.step(1)[0])
            energies.append(sv.energy())
            if k == 0:
                first = sv.get_modes()
        traj[prec] = dict(modes=sv.get_modes(), energies=energies, first=first, stats=sst)
        sv.close()
    mx, f64 = traj["mixed"], traj["fp64"]
    # the same mode count, every mode swept to the stop rules: the arithmetic alone
    fixed = dict(fixed_modes=min(6, w.M_max), als_stall_tol=args.stall)
    same = {}
    for prec in ("mixed", "fp64"):
        sv = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, prec), **fixed))
        sv.set_initial_modes(workloads.initial_modes(w))
        sv.step(1)
        same[prec] = (sv.get_modes(), sv.energy())
        sv.close()
    out["accuracy"] = {
        "steps": plan["err_steps"],
        "u_rel_l2_mixed_vs_fp64_gpu": field_rel_l2(mx["modes"], f64["modes"]),
        "energy_rel_diff_mixed_vs_fp64_gpu": abs(mx["energies"][-1] - f64["energies"][-1]) / abs(f64["energies"][-1]),
        "same_schedule": {"fixed_modes": fixed["fixed_modes"], "steps": 1,
                          "u_rel_l2_mixed_vs_fp64_gpu": field_rel_l2(same["mixed"][0], same["fp64"][0]),
                          "energy_rel_diff": abs(same["mixed"][1] - same["fp64"][1]) / abs(same["fp64"][1])},
        "energies": {k: v["energies"] for k, v in traj.items()},
        "energy_max_rel_change_per_step": {k: max((e1 - e0) / abs(e0) for e0, e1 in zip(v["energies"], v["energies"][1:]))
                                           for k, v in traj.items()},
        "modes": {k: [s["modes"] for s in v["stats"]] for k, v in traj.items()},
        "note": "both forms advanced from the initial condition under the same stop rules (free running: a mode "
                "whose amplitude sits at tol_enrich may be kept by one form and dropped by the other, so the "
                "fields agree to that truncation level); same_schedule: one step with a fixed mode count, each "
                "mode swept to the same stop rules, the arithmetic difference alone; fields compared on the "
                "nodes, rebuilt in FP64"}
    out["first_step_modes"] = {"mixed": mx["first"], "fp64": f64["first"]}
    # the precision ladder of the tensor-core contraction beside the headline's two-term split
    ladder = {}
    if args.precision == "mixed":
        for name, prec, form in (("bf16", "bf16", {}), ("split3", "split3", {}),
                                 ("split_direct_form", "mixed", dict(contraction_form=ctd.CONTRACT_DIRECT))):
            s3, t3, st3, _, _ = timed_run(ctd, torch, w, prec, plan["side_steps"], args.warmup, flush,
                                          over=dict(over, **form))
            s3.close()
            leg = leg_summary(t3, st3, w)
            leg["cube_steps"] = sum(1 for x in st3 if x.get("cube_form"))
            sv = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, prec), **fixed, **form))
            sv.set_initial_modes(workloads.initial_modes(w))
            sv.step(1)
            leg["same_schedule_u_rel_l2_vs_fp64_gpu"] = field_rel_l2(sv.get_modes(), same["fp64"][0])
            leg["same_schedule_energy_rel_diff"] = abs(sv.energy() - same["fp64"][1]) / abs(same["fp64"][1])
            sv.close()
            sv = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, prec), **over, **form))
            sv.set_initial_modes(workloads.initial_modes(w))
            energies = [sv.energy()]
            for k in range(plan["err_steps"]):
                sv.step(1)
                energies.append(sv.energy())
            leg["u_rel_l2_vs_fp64_gpu"] = field_rel_l2(sv.get_modes(), f64["modes"])
            leg["energy_rel_diff_vs_fp64_gpu"] = abs(energies[-1] - f64["energies"][-1]) / abs(f64["energies"][-1])
            leg["energy_max_rel_change_per_step"] = max((e1 - e0) / abs(e0) for e0, e1 in zip(energies, energies[1:]))
            sv.close()
            ladder[name] = leg
        ladder["note"] = ("tensor-core precisions beside the headline's hi + lo split: bf16 = one BF16 term per "
                          "factor value (1 product per K step), split3 = hi + mid + lo (6 products), "
                          "split_direct_form = the headline's split with the direct epilogue forced; each in the "
                          "automatic contraction form unless named; timed on the steps after the warm-up, errors "
                          "as in accuracy")
    out["ladder"] = ladder
    # side legs: the plain FP64 form under the same rules; both forms with the stall rule off
    side = {}
    for key, prec, o in (("fp64_same_rules", "fp64", over), ("mixed_stall_off", "mixed", dict(als_stall_tol=0.0)),
                         ("fp64_stall_off", "fp64", dict(als_stall_tol=0.0))):
        if prec == args.precision and o is over:
            continue
        s3, t3, st3, _, _ = timed_run(ctd, torch, w, prec, plan["side_steps"], args.warmup, flush, over=o)
        s3.close()
        side[key] = leg_summary(t3, st3, w)
    out["side"] = side
    return out


def single_line(w, res, args, pk, pk_kind, world, headline=True):
    """The JSON fields of one single-instance workload."""
    steps = len(res["times_ms"])
    total_ms = res["total_ms"] if "total_ms" in res else sum(res["times_ms"])
    value = replica_units(steps, world) / (total_ms / 1e3)
    key = f"{w.name}/{args.precision}"
    roof = step_roofline(w, args.precision, res["ranks_in"], res["stats"], res["times_ms"], pk, pk_kind,
                         stored_traffic(key))
    side_n = PLAN.get(w.name, dict(side_steps=2))["side_steps"]
    # the side legs time the steps right after the warm-up: compare with the same steps here
    head_leg = leg_summary(res["times_ms"][:side_n], res["stats"][:side_n], w)
    line = {"value": value, "ms_per_step": total_ms / steps, "dof_updates_per_s": value * w.grid_points,
            "modes_per_step": [s["modes"] for s in res["stats"]],
            "als_sweeps_per_step": [s["als_sweeps"] for s in res["stats"]],
            "als_stalled_per_step": [s["als_stalled"] for s in res["stats"]],
            "half_sweeps_per_s": sum(s["als_sweeps"] for s in res["stats"]) * w.dim / (total_ms / 1e3),
            "phase_us_per_half_sweep": res["phase_us_per_half_sweep"],
            "contraction_role_cycles_per_tile": res.get("contraction_role_cycles_per_tile"), "roofline": roof,
            "accuracy": res["accuracy"], "precision_ladder": res.get("ladder", {})}
    ph = res["phase_us_per_half_sweep"]
    cube_steps = sum(1 for s in res["stats"] if s.get("cube_form"))
    line["contraction_form"] = {"cube_steps": cube_steps, "direct_steps": len(res["stats"]) - cube_steps,
                                "note": "tensor-core epilogue per timed step: cube = v^3 with cbrt(c)-scaled "
                                        "columns and the exact linear part, chosen where sum_m prod_d max|a| <= "
                                        "0.6; direct = c u (u^2 - 1)"}
    if args.precision != "fp64" and ph.get("contract"):
        cr = contraction_roof_us(w, res["mk_mean"], pk, args.precision, cube_steps * 2 > len(res["stats"]))
        line["contraction_roofline"] = {
            "phase_us": ph["contract"], "roof_us": cr["roof_us"], "bound": cr["bound"],
            "frac": cr["roof_us"] / ph["contract"], "tensor_us": cr["tensor_us"], "alu_us": cr["alu_us"],
            "grid_points_of_cta": cr["grid_points"],
            "note": "the last CTA's share of one half-sweep's tensor-core contraction (phase entry to its last "
                    "tile), global-timer trace; roof = max(split MMA at one SM's share of the BF16 burst peak, "
                    "the epilogue's FP32 operations per grid point (3 direct, 2 cube form) on 128 lanes at the "
                    "maximum clock)"}
    side = dict(res["side"])
    lead = {}
    f = side.get("fp64_same_rules")
    if f and args.precision == "mixed":
        lead["per_step"] = f["ms_per_step"] / head_leg["ms_per_step"]
        lead["per_half_sweep"] = f["us_per_half_sweep"] / head_leg["us_per_half_sweep"]
    mo, fo = side.get("mixed_stall_off"), side.get("fp64_stall_off")
    if mo and fo:
        lead["per_step_stall_off"] = fo["ms_per_step"] / mo["ms_per_step"]
        lead["per_half_sweep_stall_off"] = fo["us_per_half_sweep"] / mo["us_per_half_sweep"]
    side["mixed_over_fp64_speedup"] = lead
    side["headline_same_steps"] = head_leg
    side["note"] = ("fp64_same_rules: the plain FP64 form under the headline's stop rules; *_stall_off: "
                    "tol_als and I_max only; each timed on the steps right after the same warm-up, as is "
                    "headline_same_steps (the headline's first steps), which the speedups use")
    line["compare"] = side
    return line, value


def run_gpu_main(args, rank, world, local_rank):
    import torch

    from paper_2410_15519_gb300 import build, ctd

    torch.cuda.set_device(local_rank)
    build.build()
    w = workloads.preset(args.workload, seed=workloads.preset(args.workload).seed + rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        torch.distributed.barrier()
    res = run_single(ctd, torch, w, args, flush, local_rank, headline=True)
    if world > 1:
        torch.distributed.barrier()
    res["total_ms"] = max_over_ranks(sum(res["times_ms"]), world)
    extras = {}
    if rank == 0 and world == 1:
        for name in args.extras:
            if name == args.workload:
                continue
            if name == "c4":
                extras["c4"] = run_batch(args, rank, 1, local_rank, headline=False)
            else:
                we = workloads.preset(name)
                extras[name] = (we, run_single(ctd, torch, we, args, flush, local_rank, headline=False))
    return w, res, extras


# --------------------------------------------------------------------------- batched leg (c4)
C4_COUNT, C4_SEED = 256, 4


def c4_config(ws, stall):
    sizes = {}
    for w in ws:
        sizes[w.n[0]] = sizes.get(w.n[0], 0) + 1
    return {"workload": f"c4: {len(ws)} independent 2D instances, n per dimension in "
                        f"{dict(sorted(sizes.items()))}, s=p=2, eps ~ U(0.01, 0.05), S=2, dt=1e-3, "
                        f"mode caps U{{8..40}}, rank-4 seeded cosine initial modes, tol_als=1e-08, "
                        f"als_stall_tol={stall:g}",
            "grid_points": int(sum(w.grid_points for w in ws)), "instances": len(ws),
            "l2": "no flush: the instances' operands (about 0.3 GB) exceed the 129 MB L2",
            "step": "one batched time step advances every instance by one time step"}


def run_batch(args, rank, world, local_rank, headline=True):
    """c4: every timed step is one batched launch advancing all instances by one time step."""
    import torch

    from paper_2410_15519_gb300 import build, ctd

    torch.cuda.set_device(local_rank)
    build.build()
    ws = workloads.batch_instances(C4_COUNT, C4_SEED + rank)
    over = dict(als_stall_tol=args.stall)

    def make(prec, subset=None):
        out = []
        for w in (subset if subset is not None else ws):
            s = ctd.Solver(ctd.config_from_workload(w, precision=prec_code(ctd, prec), **over))
            s.set_initial_modes(workloads.initial_modes(w))
            out.append(s)
        return out

    def timed(solvers, steps, warmup, clocks=None):
        for _ in range(warmup):
            ctd.step_batch(solvers, 1, stats=False)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        if clocks:
            clocks.start()
        stream = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctd.step_batch(solvers, steps, stats=False, stream=stream, sync=False)
        ev1.record(stream)
        ev1.synchronize()
        clk = clocks.stop() if clocks else None
        return ev0.elapsed_time(ev1), clk

    steps = args.steps if headline else args.extra_steps
    out = {"config": c4_config(ws, args.stall), "steps": steps}
    sol = make(args.precision)
    total_ms, clk = timed(sol, steps, args.warmup, ClockSampler(local_rank) if headline else None)
    if world > 1:
        torch.distributed.barrier()
    out["total_ms"] = max_over_ranks(total_ms, world)
    out["clocks"] = clk
    st = ctd.step_batch(sol, 1)
    out["sweeps_per_instance_step"] = sum(r[0]["als_sweeps"] for r in st) / len(st)
    out["modes_per_instance"] = sum(r[0]["modes"] for r in st) / len(st)
    if headline:
        # end to end: host modes of every instance in, one batched step, host modes out
        n_e2e = min(steps, 3)
        host = [s.get_modes() for s in sol]
        bi = bo = 0
        t0 = time.perf_counter()
        for k in range(n_e2e):
            for s, m in zip(sol, host):
                s.set_initial_modes(m, first_step=1000 + k)
                bi += sum(a.nbytes for a in m)
            ctd.step_batch(sol, 1, stats=False)
            host = [s.get_modes() for s in sol]
            bo += sum(a.nbytes for m in host for a in m)
        out["e2e"] = dict(steps=n_e2e, seconds=time.perf_counter() - t0, h2d=bi / n_e2e, d2h=bo / n_e2e)
    for s in sol:
        s.close()
    # accuracy: the first batched step of the smallest instances (against the oracle on the cpu leg)
    small = [w for w in ws if w.n[0] == min(x.n[0] for x in ws)][:2]
    sm = make(args.precision, small)
    ctd.step_batch(sm, 1)
    out["first_step_small"] = [(w, s.get_modes()) for w, s in zip(small, sm)]
    for s in sm:
        s.close()
    # the plain FP64 form side by side (same rules): batched, and one instance after another
    if rank == 0:
        f64 = make("fp64")
        ms64, _ = timed(f64, 1, 1)
        for s in f64:
            s.close()
        out["compare"] = {"fp64_batched_ms_per_step": ms64}
        if headline:
            seq = 0.0
            for w in ws:
                s = make("fp64", [w])[0]
                s.step(1, stats=False)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s.stream)
                s.step(1, stats=False)
                e1.record(s.stream)
                e1.synchronize()
                seq += e0.elapsed_time(e1)
                s.close()
            out["compare"]["fp64_one_instance_at_a_time_ms_per_step"] = seq
    return out


def c4_oracle_baseline(stall: float):
    """Oracle time of one batched step, estimated from one oracle step of one instance of each
    size (the batch's step time is the sum over its instances)."""
    ws = workloads.batch_instances(C4_COUNT, C4_SEED)
    per_size = {}
    for w in ws:
        if w.n[0] not in per_size:
            per_size[w.n[0]] = w
    t = {}
    for nsz, w in sorted(per_size.items()):
        code = ("import sys, time, json; sys.path.insert(0, %r)\n" % ROOT +
                "import workloads\nfrom oracle import ctd\n"
                "w = [x for x in workloads.batch_instances(%d, %d) if x.name == %r][0]\n" % (C4_COUNT, C4_SEED, w.name) +
                "prob = ctd.Problem(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, "
                "a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als, "
                "tol_enrich=w.tol_enrich, seed=w.seed, als_stall_tol=%r)\n" % stall +
                "ops = ctd.build_operators(prob); A = workloads.initial_modes(w)\n"
                "t0 = time.perf_counter(); A, st = ctd.step(prob, ops, A, 0); print(json.dumps(time.perf_counter() - t0))\n")
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], check=True, env=env, capture_output=True, text=True)
        t[nsz] = float(r.stdout.strip().splitlines()[-1])
    counts = {}
    for w in ws:
        counts[w.n[0]] = counts.get(w.n[0], 0) + 1
    batch_s = sum(counts[k] * t[k] for k in counts)
    return 1.0 / batch_s, t


def c4_first_step_errors(first, stall):
    from oracle import ctd as octd
    errs = []
    for w, G in first:
        prob = octd.Problem(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                            alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                            tol_enrich=w.tol_enrich, seed=w.seed, als_stall_tol=stall)
        ops = octd.build_operators(prob)
        A, _ = octd.step(prob, ops, workloads.initial_modes(w), 0)
        errs.append(octd.rel_l2_between(G, A))
    return errs


def batch_fields(res, world, steps):
    value = replica_units(steps, world) / (res["total_ms"] / 1e3)
    cfg = res["config"]
    out = {"value": value, "ms_per_step": res["total_ms"] / steps, "steps": steps,
           "instance_steps_per_s": value * cfg["instances"], "dof_updates_per_s": value * cfg["grid_points"],
           "sweeps_per_instance_step": res["sweeps_per_instance_step"],
           "modes_per_instance": res["modes_per_instance"], "config": cfg}
    if "compare" in res:
        c = res["compare"]
        out["compare"] = {"fp64_batched": {"ms_per_step": c["fp64_batched_ms_per_step"],
                                           "value": 1e3 / c["fp64_batched_ms_per_step"]}}
        if "fp64_one_instance_at_a_time_ms_per_step" in c:
            s = c["fp64_one_instance_at_a_time_ms_per_step"]
            out["compare"]["fp64_one_instance_at_a_time"] = {"ms_per_step": s, "value": 1e3 / s}
    return out


def main_batch(args, rank, world, local_rank):
    if args.impl == "reference":
        if rank != 0:
            return
        v, per = c4_oracle_baseline(args.stall)
        ws = workloads.batch_instances(C4_COUNT, C4_SEED)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": c4_config(ws, args.stall),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
                                 "cpu_model": cpu_model(),
                                 "sample": f"one oracle step of one instance per size {per} s, summed over the "
                                           f"batch's instances; single-threaded BLAS"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_batch(args, rank, world, local_rank)
    if rank != 0:
        return
    f = batch_fields(res, world, args.steps)
    e2e = res["e2e"]
    line = {"metric": METRIC, "value": f["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(args.precision), "data": "synthetic", "config": f["config"],
            "instance_steps_per_s": f["instance_steps_per_s"], "dof_updates_per_s": f["dof_updates_per_s"],
            "sweeps_per_instance_step": f["sweeps_per_instance_step"], "modes_per_instance": f["modes_per_instance"],
            "roofline": {"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                         "traffic": None, "kernel": "ctd::batch_step_kernel (one CTA per instance)",
                         "note": "each instance is a latency-bound chain on one SM"},
            "clocks": res["clocks"], "gpu_launches": args.steps,
            "e2e": {"value": world * e2e["steps"] / e2e["seconds"], "unit": UNIT,
                    "h2d_bytes_per_step": int(e2e["h2d"]), "d2h_bytes_per_step": int(e2e["d2h"])}}
    if "compare" in f:
        line["compare"] = f["compare"]
    if not args.no_cpu_baseline:
        v, per = c4_oracle_baseline(args.stall)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": os.cpu_count(),
                                "cpu_model": cpu_model(),
                                "sample": f"one oracle step of one instance per size {per} s, summed over the "
                                          f"batch's instances; single-threaded BLAS"}
        line["first_step_err_u_vs_oracle_smallest_instances"] = c4_first_step_errors(res["first_step_small"],
                                                                                     args.stall)
    print(json.dumps(line))


# --------------------------------------------------------------------------- main
def workload_config(w, args):
    return {"workload": f"{w.name}: {w.dim}D {'x'.join(map(str, w.n))} nodes, s={w.s} p={w.p}, eps={w.eps}, "
                        f"S={w.S}, dt={w.dt}, M_max={w.M_max}, I_max={w.I_max}, tol_als={w.tol_als}, "
                        f"als_stall_tol={args.stall:g}, tol_enrich={w.tol_enrich}",
            "grid_points": w.grid_points,
            "ic": (f"rank-{w.ic_rank} seeded cosine modes" + (" + tanh interface mode" if w.ic_tanh else "")),
            "precision": args.precision,
            "l2": "256 MB buffer written between timed steps (L2 flush)"}


def dtype_of(precision):
    rest = "; solves, Gram products, convergence test double-float (48-bit), energy FP64"
    return {"mixed": "bf16 hi+lo split (3 products)/f32-acc contraction" + rest,
            "bf16": "bf16 (1 product)/f32-acc contraction" + rest,
            "split3": "bf16 hi+mid+lo split (6 products)/f32-acc contraction" + rest,
            "fp64": "f64 contraction and energy" + rest}[precision]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=list(PRECISIONS))
    ap.add_argument("--workload", default="c3")
    ap.add_argument("--stall", type=float, default=STALL_DEFAULT,
                    help="stall rule of the fixed-point sweeps (als_stall_tol) for every leg; 0: off")
    ap.add_argument("--extras", default="c1,c2,c4",
                    help="comma-separated workloads measured after the headline and added as extra keys; none")
    ap.add_argument("--extra-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--oracle-budget", type=float, default=25.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="headline timing, phase trace and end-to-end run only (no accuracy, side or ladder legs); "
                         "for profiler captures")
    args = ap.parse_args()
    args.extras = [] if args.extras in ("", "none") else args.extras.split(",")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "c4":
        main_batch(args, rank, world, local_rank)
        return
    w = workloads.preset(args.workload)
    config = workload_config(w, args)

    if args.impl == "reference":
        if rank != 0:
            return
        budget = min(240.0, max(20.0, 4.0 * (args.steps + args.warmup)))
        info, _, res = oracle_baseline(args.workload, args.stall, budget, max_steps=args.steps + args.warmup,
                                       save=False)
        value = info["value"]
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": res["steps"], "warmup": 0, "ms_per_step": 1e3 / value, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "dof_updates_per_s": value * w.grid_points, "cpu_baseline": info,
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    wk, res, extras = run_gpu_main(args, rank, world, local_rank)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    pk, pk_kind = peaks()
    fields, value = single_line(wk, res, args, pk, pk_kind, world)
    e2e = res["e2e"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fields.pop("ms_per_step"), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(args.precision), "data": "synthetic",
            "config": config}
    line.update(fields)
    line.update({"clocks": res["clocks"], "gpu_launches": args.steps,
                 "e2e": {"value": world * e2e["steps"] / e2e["seconds"], "unit": UNIT,
                         "h2d_bytes_per_step": int(e2e["h2d"]), "d2h_bytes_per_step": int(e2e["d2h"]),
                         "steps": e2e["steps"],
                         "device_value_same_steps": e2e["steps"] / (e2e["device_ms_same_steps"] / 1e3),
                         "note": "the first timed steps again from the initial condition through the C ABI "
                                 "with host factor buffers (H2D of u^k, step, D2H of u^{k+1} each step); "
                                 "device_value_same_steps: the device-timed rate of those same steps"}})
    extra_out = {}
    for name, val in extras.items():
        if name == "c4":
            extra_out["c4"] = batch_fields(val, 1, args.extra_steps)
            continue
        we, r = val
        f, v = single_line(we, r, args, pk, pk_kind, 1, headline=False)
        f["config"] = workload_config(we, args)
        f["steps"] = len(r["times_ms"])
        extra_out[name] = f
    if not args.no_cpu_baseline:
        info, omodes, _ = oracle_baseline(args.workload, args.stall, args.oracle_budget)
        line["cpu_baseline"] = info
        if omodes is not None:
            from oracle import ctd as octd
            line["accuracy"]["first_step_err_u_vs_oracle"] = {
                k: octd.rel_l2_between(m, omodes) for k, m in res["first_step_modes"].items()}
        for name, f in extra_out.items():
            if name == "c4":
                f["first_step_err_u_vs_oracle_smallest_instances"] = c4_first_step_errors(
                    extras["c4"]["first_step_small"], args.stall)
                continue
            info, omodes, _ = oracle_baseline(name, args.stall, args.oracle_budget)
            f["cpu_baseline"] = info
            if omodes is not None:
                from oracle import ctd as octd
                f["accuracy"]["first_step_err_u_vs_oracle"] = {
                    k: octd.rel_l2_between(m, omodes) for k, m in extras[name][1]["first_step_modes"].items()}
    line["extras"] = extra_out
    print(json.dumps(line))


if __name__ == "__main__":
    main()

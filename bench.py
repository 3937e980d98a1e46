"""Benchmark: CTD Allen-Cahn time steps/s on one GB300 (and equivalent DOF-updates/s).

Default workload: 2D, 4096 x 4096 nodes (16.8M equivalent grid points), C-FEM s = p = 2,
eps = 0.01, S = 2, dt = 1e-3, up to 50 modes, seeded rank-8 cosine initial condition.  One
"step" is one full time step of the CTD solver (greedy enrichment with fixed-point sweeps and
the full-grid nonlinear contraction), launched through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--impl ours|reference]

The headline is the mixed form (split-BF16 tensor-core contraction, FP64-accurate solves,
Gram products and energy); the plain FP64 form is timed beside it ("compare").

Prints one JSON line.  Under torchrun (N > 1) every rank advances its own replica (weak
scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
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


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------------------- CPU oracle leg
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np, workloads
from oracle import ctd
w = workloads.preset({name!r})
prob = ctd.Problem(dim=w.dim, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa,
                   a0=w.a0, alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                   tol_enrich=w.tol_enrich, seed=w.seed)
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
    if steps == 1:
        np.savez({out!r} + ".npz", *A)
json.dump(dict(steps=steps, times=times, setup_s=t_setup, stats=stats), open({out!r}, "w"))
"""


def run_oracle(name: str, max_steps: int, budget_s: float):
    """Time the oracle as it stands on the host, single-threaded BLAS, in a fresh process."""
    fd, out = tempfile.mkstemp(suffix=".json")
    os.close(fd)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, budget=budget_s, max_steps=max_steps, out=out)
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


# --------------------------------------------------------------------------- GPU leg
def algorithmic_flops(w, precision: str, Mk: int, half_sweeps: int) -> float:
    """Work of the nonlinear contraction per launch (the method's own arithmetic):
    FP64 path: materialising w(u^k) (2 Mk N flops, once per step) + one FP64 multiply-add per
    grid point and half-sweep; tensor-core path: the rank-Mk reconstruction of the split
    operands, 2 (3 Mk) N per half-sweep."""
    N = float(w.grid_points)
    if precision == "fp64":
        return 2.0 * Mk * N * (w.dim - 1) + half_sweeps * 2.0 * N
    return half_sweeps * 2.0 * 3 * Mk * N


def last_cta_tile_share(w, G: int = 152) -> float:
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


def contraction_roof_us(w, Mk: float, pk: dict) -> dict:
    """Roofline time of the last CTA's share of one half-sweep's tensor-core contraction (the
    phase is timed on that CTA): the larger of the split reconstruction on the tensor cores
    (2 * 3Mk flops per grid point at one SM's share of the sustained BF16 peak) and the fused
    epilogue on the FP32 pipes (3 instructions per grid point: u*u, fma for u^3 - u, fma into
    the weighted row sum; 128 lanes x the SM clock)."""
    n_cta = float(w.grid_points) * last_cta_tile_share(w)
    t_tensor = 2.0 * 3 * Mk * n_cta / (pk["bf16_tflops_sustained"] * 1e12 / 152)
    t_alu = 3.0 * n_cta / (128 * pk.get("sm_max_mhz", 2070.0) * 1e6)
    bound = "tensor" if t_tensor >= t_alu else "alu"
    return {"roof_us": 1e6 * max(t_tensor, t_alu), "bound": bound, "tensor_us": 1e6 * t_tensor, "alu_us": 1e6 * t_alu,
            "grid_points": n_cta}


def source_hash() -> str:
    """Digest of the CUDA sources and the C ABI header (ties stored ncu counters to a build)."""
    import hashlib
    h = hashlib.sha256()
    for d in ("paper_2410_15519_gb300/csrc", "include"):
        for f in sorted(os.listdir(os.path.join(ROOT, d))):
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                h.update(f.encode())
                h.update(open(os.path.join(ROOT, d, f), "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(workload: str, precision: str):
    """DRAM bytes per launch of the step kernel from the committed ncu capture, if it was taken
    on the current sources (else None)."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")))
    except (OSError, ValueError):
        return None
    e = rec.get(f"{workload}/{precision}")
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def form_over(args, w):
    """Config overrides of the nonlinear term's form: reduced integration domain, or the
    separated form (Eq. MxySep, which takes M_max <= 16)."""
    over = dict(reduced_tol=args.reduced_tol)
    if args.nonlinear == "separated":
        over.update(nonlinear_form=1, M_max=min(w.M_max, 16))
    return over


def timed_run(ctd, torch, w, precision, steps, warmup, flush, clocks=None, over=None):
    """Advance `steps` time steps after `warmup`; one step kernel launch each, bracketed by CUDA
    events on the solver's stream, L2 flushed between steps."""
    prec = ctd.PREC_FP64 if precision == "fp64" else ctd.PREC_SPLIT_BF16
    solver = ctd.Solver(ctd.config_from_workload(w, precision=prec, **(over or {})))
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


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2410_15519_gb300 import build, ctd

    torch.cuda.set_device(local_rank)
    build.build()
    w = workloads.preset(args.workload, seed=workloads.preset(args.workload).seed + rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    over = form_over(args, w)
    solver, times_ms, stats, rank0, clk = timed_run(ctd, torch, w, args.precision, args.steps, args.warmup, flush,
                                                     clocks, over)
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(sum(times_ms), world)
    # rank of u^k entering each timed step: the previous step's output rank
    ranks_in = [rank0] + [st["modes"] for st in stats[:-1]]
    flops = sum(algorithmic_flops(w, args.precision, mk, st["als_sweeps"] * w.dim) for st, mk in zip(stats, ranks_in))
    out = dict(times_ms=times_ms, total_ms=total_ms, per_launch_ms=total_ms / args.steps, stats=stats, clocks=clk,
               flops_per_launch=flops / args.steps, mk_mean=sum(ranks_in) / len(ranks_in))
    # per-phase device time of a few more steps (global-timer trace of CTA 0)
    solver.trace(True)
    tr_steps = 3
    st_tr = solver.step(tr_steps)
    tr = solver.trace(False)
    hs = sum(s["als_sweeps"] for s in st_tr) * w.dim
    out["phase_us_per_half_sweep"] = {k: 1e6 * v / max(1, hs) for k, v in tr.items()
                                      if k in ("gram_contract", "gram", "contract", "rhs", "solve", "converge")}
    # end to end through the C ABI with host buffers: H2D of u^k, step, D2H of u^{k+1}
    n_e2e = min(args.steps, args.e2e_steps)
    modes_host = solver.get_modes()
    bi = bo = 0
    t0 = time.perf_counter()
    for k in range(n_e2e):
        bi += sum(m.nbytes for m in modes_host)
        solver.set_initial_modes(modes_host, first_step=args.warmup + args.steps + tr_steps + k)
        solver.step(1)
        modes_host = solver.get_modes()
        bo += sum(m.nbytes for m in modes_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    out["e2e"] = dict(steps=n_e2e, seconds=e2e_s, h2d=bi / max(1, n_e2e), d2h=bo / max(1, n_e2e))
    solver.close()
    # first-step result from the initial condition (accuracy check against the oracle)
    prec = ctd.PREC_FP64 if args.precision == "fp64" else ctd.PREC_SPLIT_BF16
    s2 = ctd.Solver(ctd.config_from_workload(w, precision=prec, **over))
    s2.set_initial_modes(workloads.initial_modes(w))
    s2.step(1)
    out["first_step_modes"] = s2.get_modes()
    s2.close()
    # the other arithmetic side by side (the mixed form against the plain FP64 form): its speed,
    # and both forms advanced K steps from the initial condition (field error, energy law)
    if args.compare_steps > 0 and rank == 0:
        other = "fp64" if args.precision == "mixed" else "mixed"
        s3, t3, st3, _, _ = timed_run(ctd, torch, w, other, args.compare_steps, args.warmup, flush, over=over)
        s3.close()
        traj = {}
        for prec_name in (args.precision, other):
            sv = ctd.Solver(ctd.config_from_workload(
                w, precision=ctd.PREC_FP64 if prec_name == "fp64" else ctd.PREC_SPLIT_BF16, **over))
            sv.set_initial_modes(workloads.initial_modes(w))
            energies = [sv.energy()]
            first = None
            for k in range(args.compare_steps):
                sv.step(1)
                energies.append(sv.energy())
                if k == 0:
                    first = sv.get_modes()
            traj[prec_name] = dict(modes=sv.get_modes(), energies=energies, first=first)
            sv.close()
        mixed, fp64 = traj["mixed"], traj["fp64"]
        out["compare"] = dict(precision=other, steps=len(t3), ms_per_step=sum(t3) / len(t3),
                              als_sweeps_per_step=[s["als_sweeps"] for s in st3],
                              first_step_modes=traj[other]["first"],
                              u_rel_l2_mixed_vs_fp64=sep_rel_l2(mixed["modes"], fp64["modes"]),
                              energy_rel_diff_mixed_vs_fp64=abs(mixed["energies"][-1] - fp64["energies"][-1]) /
                              abs(fp64["energies"][-1]),
                              energy_nonincreasing={k: all(e1 <= e0 + 1e-10 * abs(e0) for e0, e1 in
                                                           zip(v["energies"], v["energies"][1:]))
                                                    for k, v in traj.items()},
                              energy_first_last={k: [v["energies"][0], v["energies"][-1]] for k, v in traj.items()})
    if args.reduced_tol > 0 and args.compare_steps > 0 and rank == 0:
        sf, tf, stf, _, _ = timed_run(ctd, torch, w, args.precision, args.compare_steps, args.warmup, flush)
        sf.close()
        trajs = []
        for tol in (args.reduced_tol, 0.0):
            sv = ctd.Solver(ctd.config_from_workload(
                w, precision=ctd.PREC_FP64 if args.precision == "fp64" else ctd.PREC_SPLIT_BF16, reduced_tol=tol))
            sv.set_initial_modes(workloads.initial_modes(w))
            sv.step(args.compare_steps, stats=False)
            trajs.append(sv.get_modes())
            sv.close()
        out["full_domain"] = dict(steps=len(tf), ms_per_step=sum(tf) / len(tf),
                                  u_rel_l2_reduced_vs_full=sep_rel_l2(trajs[0], trajs[1]))
    if args.nonlinear == "separated" and args.compare_steps > 0 and rank == 0:
        # the grid form (full nodal integral on the tensor cores / in FP64) side by side
        sg, tg, stg, _, _ = timed_run(ctd, torch, w, args.precision, args.compare_steps, args.warmup, flush)
        sg.close()
        trajs = []
        for o in (over, {}):
            sv = ctd.Solver(ctd.config_from_workload(
                w, precision=ctd.PREC_FP64 if args.precision == "fp64" else ctd.PREC_SPLIT_BF16, **o))
            sv.set_initial_modes(workloads.initial_modes(w))
            sv.step(args.compare_steps, stats=False)
            trajs.append(sv.get_modes())
            sv.close()
        out["grid_form"] = dict(steps=len(tg), ms_per_step=sum(tg) / len(tg),
                                u_rel_l2_separated_vs_grid=sep_rel_l2(trajs[0], trajs[1]))
    return w, out


def sep_rel_l2(A, B):
    """Relative nodal L2 distance ||u_A - u_B|| / ||u_B|| of two separated fields (factor d of
    field X: n_d x rank array), from their grid values rebuilt in FP64 on the GPU (a Gram-matrix
    form would cancel catastrophically at the differences measured here)."""
    import torch
    def grid(X):
        t = [torch.as_tensor(x, dtype=torch.float64, device="cuda") for x in X]
        if len(t) == 2:
            return t[0] @ t[1].T
        return torch.einsum("im,jm,km->ijk", *t)
    ua, ub = grid(A), grid(B)
    return float(torch.linalg.vector_norm(ua - ub) / torch.linalg.vector_norm(ub))


# --------------------------------------------------------------------------- batched leg (c4)
C4_COUNT, C4_SEED = 256, 4


def c4_config(ws):
    sizes = {}
    for w in ws:
        sizes[w.n[0]] = sizes.get(w.n[0], 0) + 1
    return {"workload": f"c4: {len(ws)} independent 2D instances, n per dimension in "
                        f"{dict(sorted(sizes.items()))}, s=p=2, eps ~ U(0.01, 0.05), S=2, dt=1e-3, "
                        f"mode caps U{{8..40}}, rank-4 seeded cosine initial modes",
            "grid_points": int(sum(w.grid_points for w in ws)), "instances": len(ws),
            "l2": "no flush: the instances' operands (about 0.3 GB) exceed the 129 MB L2",
            "step": "one batched time step advances every instance by one time step"}


def run_batch(args, rank, world, local_rank):
    """c4: every timed step is one batched launch advancing all instances by one time step."""
    import torch

    from paper_2410_15519_gb300 import build, ctd

    torch.cuda.set_device(local_rank)
    build.build()
    ws = workloads.batch_instances(C4_COUNT, C4_SEED + rank)

    def make(prec, subset=None):
        out = []
        for w in (subset if subset is not None else ws):
            s = ctd.Solver(ctd.config_from_workload(w, precision=ctd.PREC_FP64 if prec == "fp64"
                                                    else ctd.PREC_SPLIT_BF16))
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

    out = {"config": c4_config(ws)}
    sol = make(args.precision)
    total_ms, clk = timed(sol, args.steps, args.warmup, ClockSampler(local_rank))
    if world > 1:
        torch.distributed.barrier()
    out["total_ms"] = max_over_ranks(total_ms, world)
    out["clocks"] = clk
    st = ctd.step_batch(sol, 1)
    out["sweeps_per_instance_step"] = sum(r[0]["als_sweeps"] for r in st) / len(st)
    out["modes_per_instance"] = sum(r[0]["modes"] for r in st) / len(st)
    # end to end: host modes of every instance in, one batched step, host modes out
    n_e2e = min(args.steps, 3)
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
    # accuracy: the first batched step of the smallest instances against the oracle (cpu leg)
    small = [w for w in ws if w.n[0] == min(x.n[0] for x in ws)][:2]
    sm = make(args.precision, small)
    ctd.step_batch(sm, 1)
    out["first_step_small"] = [(w, s.get_modes()) for w, s in zip(small, sm)]
    for s in sm:
        s.close()
    # the plain FP64 form side by side: batched, and one instance after another on the whole GPU
    if args.compare_steps > 0 and rank == 0:
        f64 = make("fp64")
        ms64, _ = timed(f64, 1, 1)
        for s in f64:
            s.close()
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
        out["compare"] = {"fp64_batched_ms_per_step": ms64, "fp64_one_instance_at_a_time_ms_per_step": seq}
    return out


def c4_oracle_baseline(budget_s: float):
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
                "tol_enrich=w.tol_enrich, seed=w.seed)\n"
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


def c4_first_step_errors(first):
    from oracle import ctd as octd
    errs = []
    for w, G in first:
        prob = octd.Problem(dim=2, n=w.n, length=w.length, s=w.s, p=w.p, a=w.a, L=w.L, kappa=w.kappa, a0=w.a0,
                            alpha=w.alpha, dt=w.dt, M_max=w.M_max, I_max=w.I_max, tol_als=w.tol_als,
                            tol_enrich=w.tol_enrich, seed=w.seed)
        ops = octd.build_operators(prob)
        A, _ = octd.step(prob, ops, workloads.initial_modes(w), 0)
        errs.append(octd.rel_l2_between(G, A))
    return errs


def main_batch(args, rank, world, local_rank):
    if args.impl == "reference":
        if rank != 0:
            return
        v, per = c4_oracle_baseline(args.oracle_budget)
        ws = workloads.batch_instances(C4_COUNT, C4_SEED)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": c4_config(ws),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"one oracle step of one instance per size {per} s, summed over the "
                                           f"batch's instances; single-threaded BLAS, {cpu_model()}"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res = run_batch(args, rank, world, local_rank)
    if rank != 0:
        return
    value = replica_units(args.steps, world) / (res["total_ms"] / 1e3)
    cfg = res["config"]
    e2e = res["e2e"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3-split/f32-acc; solves, Gram products, energy FP64-accurate" if args.precision == "mixed"
            else "f64", "data": "synthetic", "config": cfg,
            "instance_steps_per_s": value * cfg["instances"],
            "dof_updates_per_s": value * cfg["grid_points"],
            "sweeps_per_instance_step": res["sweeps_per_instance_step"],
            "modes_per_instance": res["modes_per_instance"],
            "roofline": {"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                         "traffic": None, "kernel": "ctd::batch_step_kernel (one CTA per instance)",
                         "note": "each instance is a latency-bound chain on one SM; see the c1 line for "
                                 "the contraction roofline"},
            "clocks": res["clocks"], "gpu_launches": args.steps,
            "e2e": {"value": world * e2e["steps"] / e2e["seconds"], "unit": UNIT,
                    "h2d_bytes_per_step": int(e2e["h2d"]), "d2h_bytes_per_step": int(e2e["d2h"])}}
    if "compare" in res:
        c = res["compare"]
        line["compare"] = {"fp64_batched": {"ms_per_step": c["fp64_batched_ms_per_step"],
                                            "value": 1e3 / c["fp64_batched_ms_per_step"]},
                           "fp64_one_instance_at_a_time": {"ms_per_step": c["fp64_one_instance_at_a_time_ms_per_step"],
                                                           "value": 1e3 / c["fp64_one_instance_at_a_time_ms_per_step"]}}
    if not args.no_cpu_baseline:
        v, per = c4_oracle_baseline(args.oracle_budget)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one oracle step of one instance per size {per} s, summed over the "
                                          f"batch's instances; single-threaded BLAS, {cpu_model()}"}
        line["first_step_err_u_vs_oracle_smallest_instances"] = c4_first_step_errors(res["first_step_small"])
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="c1")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--compare-steps", type=int, default=10,
                    help="steps of the other arithmetic (FP64 vs mixed) timed for the side-by-side numbers")
    ap.add_argument("--reduced-tol", type=float, default=0.0,
                    help="reduced integration domain: drop 128 x 128 node blocks with max |w(u^k)| <= this")
    ap.add_argument("--nonlinear", default="grid", choices=["grid", "separated"],
                    help="nonlinear term: full nodal integral (Eq. KxxMxx) or separated form (Eq. MxySep)")
    ap.add_argument("--oracle-budget", type=float, default=25.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "c4":
        main_batch(args, rank, world, local_rank)
        return
    w = workloads.preset(args.workload)
    config = {"workload": f"{w.name}: {w.dim}D {'x'.join(map(str, w.n))} nodes, s={w.s} p={w.p}, eps={w.eps}, "
                          f"S={w.S}, dt={w.dt}, M_max={w.M_max}, tol_als={w.tol_als}, tol_enrich={w.tol_enrich}",
              "grid_points": w.grid_points, "ic": (f"rank-{w.ic_rank} seeded cosine modes" + (" + tanh interface mode" if w.ic_tanh else "")),
              "precision": args.precision,
              "l2": "256 MB buffer written between timed steps (L2 flush)"}

    if args.impl == "reference":
        if rank != 0:
            return
        budget = max(10.0, 4.0 * (args.steps + args.warmup))
        res, _ = run_oracle(args.workload, args.steps + args.warmup, min(budget, 240.0))
        times = res["times"][args.warmup:] if res["steps"] > args.warmup else res["times"]
        value = len(times) / sum(times)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": len(times), "warmup": min(args.warmup, res["steps"] - len(times)),
                "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": config,
                "dof_updates_per_s": value * w.grid_points,
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"first {res['steps']} time steps of {w.name} from the initial condition, "
                                           f"single-threaded BLAS, {cpu_model()}"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    wk, res = run_gpu(args, rank, world, local_rank)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    pk, pk_kind = peaks()
    value = replica_units(args.steps, world) / (res["total_ms"] / 1e3)
    achieved = res["flops_per_launch"] / (res["per_launch_ms"] / 1e3) / 1e12
    traffic = stored_traffic(args.workload, args.precision)
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s",
                "frac": achieved / 1.25, "traffic": traffic,
                "peak_kind": "nominal FP64 rate of the part (152 SMs x 2 FP64 FMA/clk x ~2.07 GHz); "
                             "measured 1.0 TFLOP/s by a throughput probe",
                "kernel": "ctd::step_kernel (whole persistent time step)"}
        dtype = "f64"
    else:
        peak = pk["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": f"bf16 sustained, {pk_kind} (of measured)",
                "kernel": "ctd::step_kernel (whole persistent time step)"}
        dtype = "bf16x3-split/f32-acc; solves, Gram products, energy FP64-accurate"
    e2e = res["e2e"]
    ph = res["phase_us_per_half_sweep"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config,
            "dof_updates_per_s": value * wk.grid_points,
            "modes_per_step": [s["modes"] for s in res["stats"]],
            "als_sweeps_per_step": [s["als_sweeps"] for s in res["stats"]],
            "half_sweeps_per_s": sum(s["als_sweeps"] for s in res["stats"]) * wk.dim / (res["total_ms"] / 1e3),
            "phase_us_per_half_sweep": ph,
            "roofline": roof, "clocks": res["clocks"], "gpu_launches": args.steps,
            "e2e": {"value": world * e2e["steps"] / e2e["seconds"], "unit": UNIT,
                    "h2d_bytes_per_step": int(e2e["h2d"]), "d2h_bytes_per_step": int(e2e["d2h"])}}
    if args.precision == "mixed" and ph.get("contract"):
        cr = contraction_roof_us(wk, res["mk_mean"], pk)
        line["contraction_roofline"] = {
            "phase_us": ph["contract"], "roof_us": cr["roof_us"], "bound": cr["bound"],
            "frac": cr["roof_us"] / ph["contract"], "tensor_us": cr["tensor_us"], "alu_us": cr["alu_us"],
            "grid_points_of_cta": cr["grid_points"],
            "note": "the last CTA's share of one half-sweep's tensor-core contraction (phase entry to its "
                    "last tile), global-timer trace; roof = max(split MMA at one SM's share of the "
                    "sustained BF16 peak, 3 FP32 instructions per grid point on 128 lanes)"}
    if args.nonlinear == "separated":
        line["config"]["nonlinear"] = "separated (Eq. MxySep), M_max 16"
        line["roofline"] = {"bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
                            "traffic": None, "kernel": "ctd::step_kernel_sep (whole persistent time step)",
                            "note": "separated form: no grid pass and no dense phase; the step is set by its "
                                    "barriers and 1D sums (phase_us_per_half_sweep)"}
        line.pop("contraction_roofline", None)
        if "grid_form" in res:
            g = res["grid_form"]
            line["grid_form"] = {"ms_per_step": g["ms_per_step"], "value": 1e3 / g["ms_per_step"],
                                 "u_rel_l2_separated_vs_grid": g["u_rel_l2_separated_vs_grid"],
                                 "note": f"same workload with the full nodal integral, {g['steps']} steps"}
    if args.reduced_tol > 0:
        line["config"]["reduced_tol"] = args.reduced_tol
        if "full_domain" in res:
            fd = res["full_domain"]
            line["full_domain"] = {"ms_per_step": fd["ms_per_step"], "value": 1e3 / fd["ms_per_step"],
                                   "u_rel_l2_reduced_vs_full": fd["u_rel_l2_reduced_vs_full"],
                                   "note": f"same workload without the reduced domain, {fd['steps']} steps"}
    if "compare" in res:
        c = res["compare"]
        line["compare"] = {"precision": c["precision"], "steps": c["steps"], "ms_per_step": c["ms_per_step"],
                           "value": 1e3 / c["ms_per_step"], "unit": UNIT,
                           "als_sweeps_per_step": c["als_sweeps_per_step"],
                           "u_rel_l2_mixed_vs_fp64": c["u_rel_l2_mixed_vs_fp64"],
                           "energy_rel_diff_mixed_vs_fp64": c["energy_rel_diff_mixed_vs_fp64"],
                           "energy_nonincreasing": c["energy_nonincreasing"],
                           "energy_first_last": c["energy_first_last"],
                           "note": f"both forms advanced {args.compare_steps} steps from the initial condition"}
    if not args.no_cpu_baseline:
        ores, omodes = run_oracle(args.workload, 1, args.oracle_budget)
        tv = ores["steps"] / sum(ores["times"])
        line["cpu_baseline"] = {"value": tv, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {ores['steps']} time step(s) of {wk.name} from the initial "
                                          f"condition, single-threaded BLAS, {cpu_model()}"}
        if omodes is not None:
            from oracle import ctd as octd
            line["first_step_err_u_vs_oracle"] = octd.rel_l2_between(res["first_step_modes"], omodes)
            if "compare" in res:
                line["compare"]["first_step_err_u_vs_oracle"] = octd.rel_l2_between(res["compare"]["first_step_modes"],
                                                                                    omodes)
    print(json.dumps(line))


if __name__ == "__main__":
    main()

#!/usr/bin/env python
"""Benchmark: Jacobian solves per second to a 1e-8 relative residual.

Workload (one "step"): the 256x256-cell 2D log-normal permeability grid
(sigma 2, correlation length 8 cells, mean ln 1e-12), capillary scale swept over
{0, 1e3, 1e4, 1e5} Pa; for each scale the exact Newton Jacobian at the
synthetic front state is assembled on the GPU and solved by right-
preconditioned FGMRES(30) with each of the three preconditioners (black-box
AMG on J, CPR-AMG with quasi-IMPES decoupling, block factorisation with the
SIMPLE Schur complement): 12 solves per step, each with its own
preconditioner setup. V-cycles run in FP64 for the headline number (the
workload's "plain FP64 on GPU"); the same step with FP32 V-cycles is reported
beside it. A solve counts when its true relative residual is <= 1e-8 within
`--maxit` Arnoldi steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs the same step on its own GPU (replicas;
no data-path collective) and `value` is all ranks' solves over the slowest
rank's time. `--impl reference` times the CPU oracle on a bounded sample of
the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

METRIC = "Jacobian solves/s to 1e-8 relative residual (256x256 2D log-normal, 4 capillary scales x 3 preconditioners)"
UNIT = "solves/s"
WORKLOAD = "2d_256x256_lognormal_sigma2_ell8_pc{0,1e3,1e4,1e5}_x_{amgJ,cpr1_qimpes,bf}"
PC_SCALES = (0.0, 1e3, 1e4, 1e5)
KINDS = (("amgJ", 0, 0), ("cpr1", 1, 2), ("bf", 3, 0))
# DRAM bytes (read + write) per launch of the roofline kernels, from one ncu
# capture of the current kernel version (summaries and commands in profiles/);
# None where no capture of the current version exists.
NCU_TRAFFIC = {
    ("k_hgs", "fp64", "lognormal256bf"): (11.765248e6 + 0.0, "profiles/k_hgs_fp64_lognormal256_bf_level0.md"),
    ("k_hgs", "fp64", "layered128"): (225.423104e6 + 11.490048e6, "profiles/k_hgs_fp64_layered128_level0.md"),
    ("k_bsr2_spmv", "f64", "layered128"): (608.675840e6 + 30.454272e6, "profiles/k_bsr2_spmv_layered128.md"),
    ("k_hgs", "fp32", "layered128"): (150.313472e6 + 6.125056e6, "profiles/k_hgs_fp32_layered128_level0.md"),
    ("k_csr_residual", "fp32", "layered128"): (142.222336e6 + 4.032768e6,
                                             "profiles/k_csr_residual_fp32_layered128_level0.md"),
    ("k_csr_restrict", "fp32", "layered128"): (60.598272e6 + 0.020992e6,
                                             "profiles/k_csr_restrict_fp32_layered128_level0.md"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    return ap.parse_args()


def workload(n):
    from paper_1611_00127_gb300 import inputs as I
    probs, states = [], []
    for pc in PC_SCALES:
        p = I.config_lognormal_2d(pc, n=n)
        probs.append(p)
        states.append(I.front_state(p))
    return probs, states


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ GPU arm
class GpuStep:
    def __init__(self, probs, states, precision, maxit):
        import torch
        from paper_1611_00127_gb300 import rsflow as R
        self.R, self.torch = R, torch
        self.probs = probs
        self.precision = precision
        self.maxit = maxit
        self.dps = [R.DeviceProblems(p) for p in probs]
        self.J = R.Bsr2.pattern(self.dps[0])
        n = 2 * probs[0].ncell
        self.n = n
        self.F = torch.empty(n, dtype=torch.float64, device="cuda")
        self.b = torch.empty(n, dtype=torch.float64, device="cuda")
        self.x = torch.empty(n, dtype=torch.float64, device="cuda")
        self.u = [torch.as_tensor(s[0], device="cuda") for s in states]
        self.uo = [torch.as_tensor(s[1], device="cuda") for s in states]
        self.xout = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(len(probs) * len(KINDS))]
        # pick the block SpMV's lanes per row for this matrix (autotuner)
        R.jacobian_assemble(self.dps[0], self.u[0], self.uo[0], 86400.0, self.J, self.F)
        self.lanes = R.autotune_bsr2(self.J, self.F, self.x)

    def params(self, kind, dec):
        R = self.R
        return R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=self.precision))

    def run(self, dps=None, us=None, uos=None, per_solve_profile=None):
        """One step; returns per-solve records. With `per_solve_profile` (a
        dict), each solve runs between profile_begin/profile_end and its
        kernel-class times are stored under the solve's name."""
        R, torch = self.R, self.torch
        dps = dps or self.dps
        us = us or self.u
        uos = uos or self.uo
        recs = []
        q = 0
        for k in range(len(self.probs)):
            R.jacobian_assemble(dps[k], us[k], uos[k], 86400.0, self.J, self.F)
            torch.neg(self.F, out=self.b)
            for name, kind, dec in KINDS:
                tag = f"pc{PC_SCALES[k]:g}_{name}"
                torch.cuda.nvtx.range_push(tag)
                if per_solve_profile is not None:
                    torch.cuda.synchronize()
                    R.profile_begin()
                self.xout[q].zero_()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                ev[0].record()
                M = R.Precond(self.J, self.params(kind, dec))
                ev[1].record()
                st = R.gmres_solve(self.J, M, self.b, self.xout[q], R.GmresParams(m=30, maxit=self.maxit, rtol=1e-8))
                ev[2].record()
                M.close()
                if per_solve_profile is not None:
                    torch.cuda.synchronize()
                    per_solve_profile[tag] = R.profile_end()
                torch.cuda.nvtx.range_pop()
                ev[2].synchronize()
                recs.append(dict(pc=PC_SCALES[k], prec=name, its=int(st.iterations), relres=float(st.relres),
                                 converged=bool(st.converged == 1), setup_ms=round(ev[0].elapsed_time(ev[1]), 3),
                                 solve_ms=round(ev[1].elapsed_time(ev[2]), 3)))
                q += 1
        return recs


class GpuBatchStep:
    """The same 12 solves as a batch: the four Jacobians stacked block-diagonally
    (one assembly call), one preconditioner setup and one FGMRES call per kind
    for all four systems (segment-indexed kernels, per-system convergence)."""

    def __init__(self, probs, states, precision, maxit):
        import torch
        from paper_1611_00127_gb300 import rsflow as R
        self.R, self.torch = R, torch
        self.probs = probs
        self.precision = precision
        self.maxit = maxit
        self.dp = R.DeviceProblems(probs)
        self.J = R.Bsr2.pattern(self.dp)
        n = 2 * self.dp.ncell
        self.F = torch.empty(n, dtype=torch.float64, device="cuda")
        self.b = torch.empty(n, dtype=torch.float64, device="cuda")
        self.u = torch.as_tensor(np.concatenate([s[0] for s in states]), device="cuda")
        self.uo = torch.as_tensor(np.concatenate([s[1] for s in states]), device="cuda")
        self.xout = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in KINDS]

    def run(self):
        R = self.R
        R.jacobian_assemble(self.dp, self.u, self.uo, 86400.0, self.J, self.F)
        self.torch.neg(self.F, out=self.b)
        recs = []
        for q, (name, kind, dec) in enumerate(KINDS):
            self.xout[q].zero_()
            M = R.Precond(self.J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=self.precision)))
            st = R.gmres_solve(self.J, M, self.b, self.xout[q], R.GmresParams(m=30, maxit=self.maxit, rtol=1e-8))
            M.close()
            for k in range(len(self.probs)):
                recs.append(dict(pc=PC_SCALES[k], prec=name, its=int(st.its[k]), relres=float(st.relres_seg[k]),
                                 converged=bool(st.relres_seg[k] <= 1e-8)))
        return recs


def flush_l2(buf):
    buf.add_(1.0)


def hbm_peak():
    """Measured STREAM-copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sweep_roofline(probs, states, precision, reps=50):
    """Average device duration of the dominant kernel (one hybrid Gauss-Seidel
    sweep of level 0 of the largest hierarchy in the workload: the SIMPLE Schur
    complement of the block-factorisation preconditioner at capillary scale
    1e3), timed with CUDA events on the launching stream over `reps`
    back-to-back launches, and the block SpMV timed the same way."""
    from paper_1611_00127_gb300 import kernel_bench
    from paper_1611_00127_gb300 import rsflow as R
    return kernel_bench.lognormal(probs[1].nx, PC_SCALES[1], precision, R.BF, reps)


def sweep_roofline_3d(precision, n=128, reps=20):
    """The same sweep on an HBM-resident case: level 0 (A_pp, 2.1M rows) of the
    CPR hierarchy of the 128^3 layered workload, L2 flushed before the loop."""
    from paper_1611_00127_gb300 import kernel_bench
    from paper_1611_00127_gb300 import rsflow as R
    return kernel_bench.layered(n, precision, R.CPR1, reps)


def shares(prof):
    tot = sum(v[0] for v in prof.values()) or 1.0
    return {k: round(v[0] / tot, 4) for k, v in prof.items() if v[2] > 0}


def profiled_step(step):
    """One more step with the library's event profiling on, solve by solve:
    per kernel class device time, algorithmic bytes and launches (the
    preconditioner applies run without graph replay so every launch is
    timed). Returns (whole-step totals, per-solve classes)."""
    import torch
    per = {}
    torch.cuda.synchronize()
    step.run(per_solve_profile=per)
    tot = {}
    for prof in per.values():
        for k, (ms, by, n) in prof.items():
            a = tot.get(k, (0.0, 0.0, 0))
            tot[k] = (a[0] + ms, a[1] + by, a[2] + n)
    return tot, per


def time_steps(step, steps, warmup, sync_barrier):
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(warmup):
        step.run()
    torch.cuda.synchronize()
    total_ms = 0.0
    recs = None
    for _ in range(steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        sync_barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("step")
        e0.record()
        recs = step.run()
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        total_ms += e0.elapsed_time(e1)
    return total_ms, recs


def e2e_steps(probs, states, precision, maxit, steps, warmup):
    """The same step through the public API starting from pinned host inputs:
    permeability fields and states copied in, every solution copied out,
    inside the timed region."""
    import torch
    from paper_1611_00127_gb300 import rsflow as R
    n = 2 * probs[0].ncell
    host_k = [torch.from_numpy(np.ascontiguousarray(np.stack([p.kx, p.ky, p.kz]))).pin_memory() for p in probs]
    host_u = [torch.from_numpy(np.ascontiguousarray(s[0])).pin_memory() for s in states]
    host_uo = [torch.from_numpy(np.ascontiguousarray(s[1])).pin_memory() for s in states]
    host_x = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(len(probs) * len(KINDS))]
    step = GpuStep(probs, states, precision, maxit)
    dev_k = [torch.empty_like(h, device="cuda") for h in host_k]
    dev_u = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in probs]
    dev_uo = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in probs]
    # problems bound to the device buffers that the copies refill every step
    dps = []
    for k, p in enumerate(probs):
        dp = R.DeviceProblems(p)
        dp.c[0].kx, dp.c[0].ky, dp.c[0].kz = (dev_k[k][0].data_ptr(), dev_k[k][1].data_ptr(), dev_k[k][2].data_ptr())
        dps.append(dp)
    h2d = sum(h.numel() * 8 for h in host_k) + sum(h.numel() * 8 for h in host_u) * 2
    d2h = sum(h.numel() * 8 for h in host_x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def one():
        for k in range(len(probs)):
            dev_k[k].copy_(host_k[k], non_blocking=True)
            dev_u[k].copy_(host_u[k], non_blocking=True)
            dev_uo[k].copy_(host_uo[k], non_blocking=True)
        recs = step.run(dps, dev_u, dev_uo)
        for q, h in enumerate(host_x):
            h.copy_(step.xout[q], non_blocking=True)
        return recs

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    total = 0.0
    nconv = 0
    for _ in range(steps):
        flush.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs = one()
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
        nconv += sum(r["converged"] for r in recs)
    return nconv, total, h2d, d2h


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(probs, states, maxit, budget_s=20.0):
    """Times the oracle (single-threaded, as it stands) on whole solves of the
    same workload, in workload order, until ~budget_s of CPU time is used."""
    import oracle as O
    t0 = time.perf_counter()
    done, conv, ran = 0, 0, []
    for k, p in enumerate(probs):
        F, J, (rp, col) = O.assemble(p, states[k][0], states[k][1], 86400.0)
        for name, kind, dec in KINDS:
            M = O.Precond(rp, col, J, O.PrecParams(kind=kind, decouple=dec))
            x, st, its, rr = O.fgmres(rp, col, J, -F, M, m=30, rtol=1e-8, maxit=maxit)
            done += 1
            conv += int(st == 0)
            ran.append(f"pc{PC_SCALES[k]:g}/{name}")
            if time.perf_counter() - t0 > budget_s:
                break
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return dict(value=conv / el, unit=UNIT, cores=1, kind="oracle",
                sample=f"{done} of 12 solves of one step ({', '.join(ran)}), {conv} converged, {el:.1f} s, "
                       f"assembly + setup + FGMRES per solve")


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    probs, states = workload(args.n)
    import oracle as O
    O.build()
    vals, samples = [], []
    for w in range(args.warmup + args.steps):
        # each step: one bounded sample (first solves of the workload, ~10 s)
        r = oracle_sample(probs, states, args.maxit, budget_s=10.0)
        if w >= args.warmup:
            vals.append(r["value"])
            samples.append(r["sample"])
    v = float(np.mean(vals))
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=None, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, grid=f"{args.n}x{args.n}", solves_per_step=12,
                            gmres="FGMRES(30), rtol 1e-8, maxit %d" % args.maxit, vcycle="FP64",
                            parallelism="single host core"),
                cpu_baseline=dict(value=v, unit=UNIT, cores=1, kind="oracle", sample=samples[-1]),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def ensemble_bench(maxit):
    """The 96-member ensemble (2D grids with sides 64..512, each its own
    log-normal field; one Jacobian each at the front state): CPR-AMG(1)
    FGMRES to 1e-8 (at most `maxit` iterations), timed (set-up + solve, L2 flushed before each form) as
    (a) 96 single-system solves with FP64 V-cycles one after another and
    (b) one batched solve with FP32 V-cycles: one set-up and one FGMRES call
    over the 96 stacked systems. One untimed run of each form first."""
    import torch
    from paper_1611_00127_gb300 import inputs as I
    from paper_1611_00127_gb300 import rsflow as R
    probs = I.config_ensemble()
    states = [I.front_state(p) for p in probs]
    singles = []
    for p, (u, uo) in zip(probs, states):
        dp = R.DeviceProblems(p)
        J = R.Bsr2.pattern(dp)
        F = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
        R.jacobian_assemble(dp, torch.as_tensor(u, device="cuda"), torch.as_tensor(uo, device="cuda"), I.DAY, J, F)
        singles.append((J, F))
    dpb = R.DeviceProblems(probs)
    Jb = R.Bsr2.pattern(dpb)
    Fb = torch.empty(2 * dpb.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dpb, torch.as_tensor(np.concatenate([s[0] for s in states]), device="cuda"),
                        torch.as_tensor(np.concatenate([s[1] for s in states]), device="cuda"), I.DAY, Jb, Fb)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    gp = R.GmresParams(maxit=maxit)

    def single_run():
        conv = 0
        for J, F in singles:
            M = R.Precond(J, R.PrecParams(kind=R.CPR1, amg=R.AmgParams(precision=R.FP64)))
            x = torch.zeros_like(F)
            st = R.gmres_solve(J, M, -F, x, gp)
            conv += int(st.converged)
            M.close()
        return conv

    def batched_run():
        M = R.Precond(Jb, R.PrecParams(kind=R.CPR1, amg=R.AmgParams(precision=R.FP32)))
        x = torch.zeros_like(Fb)
        st = R.gmres_solve(Jb, M, -Fb, x, gp)
        M.close()
        return int(st.converged)

    out = {}
    for name, fn in (("fp64_single", single_run), ("fp32_batched", batched_run)):
        fn()
        flush_l2(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        conv = fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = dict(ms=ms, converged=conv, solves_per_s=conv / (ms * 1e-3) if ms > 0 else None)
    f64, f32 = out["fp64_single"], out["fp32_batched"]
    return dict(members=len(probs), cells=int(dpb.ncell), preconditioner="CPR-AMG(1), quasi-IMPES",
                fp64_single=f64, fp32_batched=f32,
                speedup=(f32["solves_per_s"] / f64["solves_per_s"]) if f64["solves_per_s"] else None,
                how="set-up + FGMRES to 1e-8, CUDA events, L2 flushed before each timed form")


def reduce_over_ranks(times_ms, converged, dist, device):
    """Whole-job figures of a replicated step: the slowest rank's times (MAX)
    and the converged solves of all ranks (SUM). With dist None (one
    process) the inputs come back unchanged."""
    import torch
    if dist is None:
        return list(times_ms), list(converged)
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    c = torch.tensor(list(converged), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(v) for v in t], [int(round(float(v))) for v in c]


def solves_per_second(converged, steps, total_ms):
    """Converged solves of all ranks over the slowest rank's time."""
    return converged * steps / (total_ms / 1e3) if total_ms > 0 else 0.0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1611_00127_gb300 import rsflow as R
    probs, states = workload(args.n)
    R.lib()
    # headline: FP64 V-cycles
    step64 = GpuStep(probs, states, R.FP64, args.maxit)
    l0 = R.launch_count()
    with ClockSampler(local) as clk:
        ms64, recs64 = time_steps(step64, args.steps, args.warmup, barrier)
    launches = (R.launch_count() - l0)
    conv64 = sum(r["converged"] for r in recs64)
    step32 = GpuStep(probs, states, R.FP32, args.maxit)
    ms32, recs32 = time_steps(step32, args.steps, 1, barrier)
    conv32 = sum(r["converged"] for r in recs32)
    stepb = GpuBatchStep(probs, states, R.FP32, args.maxit)
    msb, recsb = time_steps(stepb, args.steps, 1, barrier)
    convb = sum(r["converged"] for r in recsb)
    (ms64, ms32, msb), (conv64, conv32, convb) = reduce_over_ranks([ms64, ms32, msb], [conv64, conv32, convb],
                                                                   dist, "cuda")
    value = solves_per_second(conv64, args.steps, ms64)
    value32 = solves_per_second(conv32, args.steps, ms32)
    valueb = solves_per_second(convb, args.steps, msb)
    e2e = None
    if not args.no_e2e:
        nconv_e, total_s, h2d, d2h = e2e_steps(probs, states, R.FP64, args.maxit, args.steps, 1)
        (te_ms,), (ce,) = reduce_over_ranks([total_s * 1e3], [nconv_e], dist, "cuda")
        e2e = dict(value=solves_per_second(ce, 1, te_ms), unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h)
    if rank != 0:
        return
    prof, per_solve = profiled_step(step64)
    peak, peak_kind = hbm_peak()
    rl = sweep_roofline(probs, states, R.FP64)
    achieved = rl["sweep_bytes"] / (rl["sweep_ms"] * 1e-3) / 1e9
    roofline = dict(bound="hbm", kernel="k_hgs (hybrid multicolour Gauss-Seidel sweep, FP64)",
                    achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                    traffic=NCU_TRAFFIC[("k_hgs", "fp64", "lognormal256bf")][0],
                    traffic_source=NCU_TRAFFIC[("k_hgs", "fp64", "lognormal256bf")][1] + " (caches flushed by ncu)",
                    peak_source=peak_kind, launch_ms=rl["sweep_ms"], bytes_per_launch=rl["sweep_bytes"],
                    units=f"level 0 of the Schur-complement hierarchy: {rl['rows']} rows, {rl['nnz']} entries",
                    note="working set of this 256x256 workload is L2-resident (<129 MB); roofline_large repeats "
                         "the measurement on an HBM-resident 128^3 level")
    roofline_large = None
    if not args.no_large:
        roofline_large = {}
        for pname, prec in (("fp64", R.FP64), ("fp32", R.FP32)):
            big = sweep_roofline_3d(prec)
            a2 = big["sweep_bytes"] / (big["sweep_ms"] * 1e-3) / 1e9
            s2 = big["spmv_bytes"] / (big["spmv_ms"] * 1e-3) / 1e9
            tr, src = NCU_TRAFFIC.get(("k_hgs", pname, "layered128"), (None, None))
            trs, srcs = NCU_TRAFFIC.get(("k_bsr2_spmv", "f64", "layered128"), (None, None))
            roofline_large[pname] = dict(
                bound="hbm", kernel=f"k_hgs {pname.upper()}, level 0 (A_pp) of the 128^3 layered CPR hierarchy",
                achieved=a2, peak=peak, unit="GB/s", frac=a2 / peak, traffic=tr, traffic_source=src,
                launch_ms=big["sweep_ms"], bytes_per_launch=big["sweep_bytes"],
                units=f"{big['rows']} rows, {big['nnz']} entries",
                bsr2_spmv=dict(achieved=s2, frac=s2 / peak, launch_ms=big["spmv_ms"], traffic=trs,
                               traffic_source=srcs, bytes_per_launch=big["spmv_bytes"], nnzb=big["nnzb"]),
                transfer={k: dict(achieved=v["gbs"], frac=v["gbs"] / peak, launch_ms=v["ms"],
                              bytes_per_launch=v["bytes"],
                              traffic=NCU_TRAFFIC.get(("k_csr_" + k, pname, "layered128"), (None,))[0])
                          for k, v in big["transfer"].items()},
                l2="flushed before the timed launches; working set > L2")
    spmv = dict(achieved=rl["spmv_bytes"] / (rl["spmv_ms"] * 1e-3) / 1e9, launch_ms=rl["spmv_ms"],
                bytes_per_launch=rl["spmv_bytes"])
    kernel_profile = {k: dict(ms=v[0], gbs=(v[1] / (v[0] * 1e-3) / 1e9 if v[0] > 0 else 0.0), launches=v[2])
                      for k, v in prof.items() if v[2] > 0}
    ensemble = None if args.no_ensemble else ensemble_bench(600)
    cpu = None if args.no_cpu_baseline else oracle_sample(probs, states, args.maxit)
    warmup_launch_note = "counted over warm-up + timed steps / (warm-up + timed)"
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms64 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
        data="synthetic",
        config=dict(workload=WORKLOAD, grid=f"{args.n}x{args.n}", solves_per_step=12,
                    bsr2_lanes_per_row=step64.lanes,
                    converged_per_step=conv64, gmres="FGMRES(30), rtol 1e-8, maxit %d" % args.maxit,
                    vcycle="FP64", l2="flushed (256 MB write) before every timed step",
                    parallelism="replicas" if world > 1 else "single GPU"),
        solves=recs64,
        fp32_vcycle=dict(value=value32, ms_per_step=ms32 / args.steps, converged_per_step=conv32, solves=recs32),
        batched_fp32=dict(value=valueb, ms_per_step=msb / args.steps, converged_per_step=convb,
                          speedup_vs_fp64_single=valueb / value if value > 0 else None,
                          how="4 Jacobians stacked as one batch; one setup + one FGMRES call per preconditioner kind",
                          solves=recsb),
        clocks=clk.summary(),
        roofline=roofline,
        roofline_large=roofline_large,
        ensemble=ensemble,
        bsr2_spmv=spmv,
        kernel_profile=dict(note="one eager profiled step, CUDA events per launch (includes launch gaps)",
                            classes=kernel_profile,
                            shares_pc10000_cpr1=shares(per_solve.get("pc10000_cpr1", {}))),
        gpu_launches=int(round(launches / (args.steps + args.warmup))) * args.steps,
        e2e=e2e,
        cpu_baseline=cpu,
    )
    print(json.dumps(line))


if __name__ == "__main__":
    main()

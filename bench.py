#!/usr/bin/env python
"""Benchmark: Jacobian solves per second to a 1e-8 relative residual.

Headline workload (one "step"): the 256^3-cell 3D channelised grid (33.5M
unknowns; 30 % channel facies from a Gaussian field with correlation lengths
64/8/4 cells, k = 1e-11 in channels and 1e-15 outside, times a unit log-normal
noise; Brooks-Corey entry pressure 1e4 Pa) at the first Newton iterate of its
first one-day backward-Euler step. Each step assembles F and the exact
Jacobian J on the GPU and solves J dx = -F twice, with CPR-AMG (quasi-IMPES
decoupling, Alg. 1) and with block factorisation (SIMPLE Schur complement,
Alg. 3), each from its own preconditioner set-up: right-preconditioned
FGMRES(30) in FP64 with FP32 V-cycles, to a true relative residual of 1e-8.
A solve counts when it converges within `--maxit` Arnoldi steps; solves/s is
converged solves over the wall time of assembly + set-ups + solves.

Beside it, on one GPU: the same step with FP64 V-cycles; the 128^3 layered
grid with FP32 and FP64 V-cycles; the 256x256 log-normal grid (12 solves:
4 capillary scales x 3 preconditioners) single-system and batched; the
96-member ensemble; the level-0 kernels of the 256^3 hierarchy against the
HBM roofline; the same step end to end from host buffers; and the CPU
oracle on a bounded window of the same field.

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

METRIC = "Jacobian solves/s to 1e-8 relative residual"
UNIT = "solves/s"
WORKLOAD = "3d_256^3_channel_first_newton_jacobian_x_{cpr1_qimpes,bf}_fp32_vcycle"
WORKLOAD_2D = "2d_256x256_lognormal_sigma2_ell8_pc{0,1e3,1e4,1e5}_x_{amgJ,cpr1_qimpes,bf}"
PC_SCALES = (0.0, 1e3, 1e4, 1e5)
KINDS = (("amgJ", 0, 0), ("cpr1", 1, 2), ("bf", 3, 0))
KINDS_3D = (("cpr1", 1, 2), ("bf", 3, 0))
THETA_3D = 0.5
# the CPU oracle's window of the 256^3 field: the corner block of this many
# cells (1/128 of the grid)
WINDOW = (64, 64, 32)
# DRAM bytes (read + write) of all launches of a kernel class in one headline
# step, from an ncu capture of the current kernels on the 128^3 grid of the
# same generator scaled to 256^3 by the cell ratio 8 (summary and command in
# profiles/dram_setup_channel128_step.md); absent where no capture of the
# current version exists.
NCU_TRAFFIC = {
    "setup_spgemm": ((41.395e9 + 12.701e9) * 8, "profiles/dram_setup_channel128_step.md (128^3 step x 8)"),
    "setup_interp": ((8.074e9 + 0.805e9) * 8, "profiles/dram_setup_channel128_step.md (128^3 step x 8)"),
}
# nominal HBM3e bandwidth of a GB300 (the fractions are also given against it)
NOMINAL_HBM_GBS = 7900.0
# the kernels behind each class of the library's event profiler
CLASS_KERNELS = {
    "setup_spgemm": "k_spgemm_bin1, k_spgemm_binfill, k_spgemm, k_copy_rows (Galerkin and Schur-complement "
                    "sparse products)",
    "setup_interp": "k_interp_ext_w (extended+i interpolation weights)",
    "hybrid_gs_sweep": "k_hgs, k_hgs2 (hybrid Gauss-Seidel sweeps)",
    "csr_resid_restrict_prolong": "k_csr (residual, restriction, prolongation)",
    "bsr2_spmv": "k_bsr2_spmv, k_cpr_resid (block SpMV)",
    "gmres_cgs2": "k_arnoldi (CGS2 passes)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--n3", type=int, default=256, help="cells per side of the 3D channelised headline grid")
    ap.add_argument("--n", type=int, default=256, help="cells per side of the 2D log-normal grid")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-side", action="store_true", help="headline legs only (no 128^3, 2D, ensemble legs)")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline timing only: no FP64 leg, end-to-end leg, profiled step, level-0 kernels, "
                         "side legs or CPU baseline (for profiler launch lists)")
    ap.add_argument("--newton", action="store_true",
                    help="also run the full Newton sequence (5 one-day steps) on the headline grid")
    return ap.parse_args()


def restriction_2d(kind):
    """Restriction of the scalar hierarchies on the 2D log-normal workload:
    block factorisation (kind 3) takes the localised approximate ideal
    restriction, under which its A_ss and Schur-complement V-cycles converge
    at capillary scales 1e4 and 1e5 where the Galerkin ones stall; the other
    kinds, and every kind on the 3D workloads, keep the Galerkin R = P^T."""
    return 3 if kind == 3 else 0


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
        return R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=self.precision,
                                                                     restriction=restriction_2d(kind)))

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
            M = R.Precond(self.J, R.PrecParams(kind=kind, decouple=dec,
                                               amg=R.AmgParams(precision=self.precision,
                                                               restriction=restriction_2d(kind))))
            st = R.gmres_solve(self.J, M, self.b, self.xout[q], R.GmresParams(m=30, maxit=self.maxit, rtol=1e-8))
            M.close()
            for k in range(len(self.probs)):
                recs.append(dict(pc=PC_SCALES[k], prec=name, its=int(st.its[k]), relres=float(st.relres_seg[k]),
                                 converged=bool(st.relres_seg[k] <= 1e-8)))
        return recs


class Gpu3DStep:
    """One step of a 3D workload: assemble F and J at the first Newton iterate
    of the first time step (u = u_old = the initial state), then for each
    preconditioner kind a set-up and an FGMRES(30) solve of J dx = -F to 1e-8
    from dx = 0. With `host` (pinned host copies of kx, ky, kz and u), every
    step first copies the inputs to the device and every solution back."""

    def __init__(self, p, precision, maxit, host=None):
        import torch
        from paper_1611_00127_gb300 import inputs as I
        from paper_1611_00127_gb300 import rsflow as R
        self.R, self.torch, self.I = R, torch, I
        self.p = p
        self.precision = precision
        self.maxit = maxit
        self.dp = R.DeviceProblems(p)
        self.J = R.Bsr2.pattern(self.dp)
        n = 2 * p.ncell
        self.F = torch.empty(n, dtype=torch.float64, device="cuda")
        self.b = torch.empty(n, dtype=torch.float64, device="cuda")
        self.u = torch.as_tensor(I.initial_state(p), device="cuda")
        self.xout = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in KINDS_3D]
        self.host = host
        self.hier = {}   # per preconditioner: its hierarchies (filled by a profiled step)
        if host is not None:
            # the problem reads its permeability from buffers the copies refill
            self.dk = torch.empty_like(host["k"], device="cuda")
            self.dp.c[0].kx, self.dp.c[0].ky, self.dp.c[0].kz = (self.dk[0].data_ptr(), self.dk[1].data_ptr(),
                                                                 self.dk[2].data_ptr())
            self.hx = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in KINDS_3D]
            self.h2d = host["k"].numel() * 8 + host["u"].numel() * 8
            self.d2h = sum(h.numel() * 8 for h in self.hx)

    def params(self, kind, dec):
        R = self.R
        return R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(theta=THETA_3D, precision=self.precision))

    def run(self, per_solve_profile=None):
        R, torch = self.R, self.torch
        if self.host is not None:
            self.dk.copy_(self.host["k"], non_blocking=True)
            self.u.copy_(self.host["u"], non_blocking=True)
        R.jacobian_assemble(self.dp, self.u, self.u, self.I.DAY, self.J, self.F)
        torch.neg(self.F, out=self.b)
        recs = []
        for q, (name, kind, dec) in enumerate(KINDS_3D):
            torch.cuda.nvtx.range_push(name)
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
            if per_solve_profile is not None:
                try:
                    self.hier[name] = hierarchy_stats(M)
                except Exception as e:   # a report field only: never fail the bench on it
                    self.hier[name] = dict(error=str(e))
            M.close()
            if per_solve_profile is not None:
                torch.cuda.synchronize()
                per_solve_profile[name] = R.profile_end()
            torch.cuda.nvtx.range_pop()
            if self.host is not None:
                self.hx[q].copy_(self.xout[q], non_blocking=True)
            ev[2].synchronize()
            recs.append(dict(prec=name, its=int(st.iterations), relres=float(st.relres),
                             converged=bool(st.converged == 1), setup_ms=round(ev[0].elapsed_time(ev[1]), 3),
                             solve_ms=round(ev[1].elapsed_time(ev[2]), 3)))
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


def shares(prof):
    tot = sum(v[0] for v in prof.values()) or 1.0
    return {k: round(v[0] / tot, 4) for k, v in prof.items() if v[2] > 0}


def hierarchy_stats(M):
    """Levels, rows per level and operator complexity (the levels' nonzeros
    summed over the finest level's) of each AMG hierarchy inside a
    preconditioner (which 0: pressure block, Schur complement or black-box;
    1: the saturation block)."""
    out = {}
    for which, name in ((0, "hierarchy_0"), (1, "hierarchy_1")):
        H = M.amg(which)
        if H is None:
            continue
        info = [H.level_info(l) for l in range(H.nlevels)]
        nnz0 = info[0][1] if info and info[0][1] > 0 else 1
        out[name] = dict(levels=len(info), rows=[x[0] for x in info],
                         op_complexity=sum(x[1] for x in info) / nnz0)
    return out


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
    """W untimed steps, then K steps each bracketed by an L2 flush, a barrier
    and a device synchronisation and timed with CUDA events. Returns (total
    ms, last step's records, launches of the library's kernels in the timed
    steps)."""
    import torch
    from paper_1611_00127_gb300 import rsflow as R
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(warmup):
        step.run()
    torch.cuda.synchronize()
    total_ms = 0.0
    recs = None
    launches = 0
    for _ in range(steps):
        flush_l2(flush)
        torch.cuda.synchronize()
        sync_barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("step")
        l0 = R.launch_count()
        e0.record()
        recs = step.run()
        e1.record()
        torch.cuda.synchronize()
        launches += R.launch_count() - l0
        torch.cuda.nvtx.range_pop()
        total_ms += e0.elapsed_time(e1)
    return total_ms, recs, launches


def e2e_wall(step, steps, warmup):
    """Wall-clock time of `steps` steps of a host-buffer step (inputs copied
    in and solutions copied out inside each step), after `warmup` steps."""
    import torch
    for _ in range(warmup):
        step.run()
    torch.cuda.synchronize()
    total, nconv = 0.0, 0
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        recs = step.run()
        torch.cuda.synchronize()
        total += time.perf_counter() - t0
        nconv += sum(r["converged"] for r in recs)
    return nconv, total


# ------------------------------------------------------------------ CPU oracle
def oracle_window(p_full, maxit, its_full=None):
    """The CPU oracle (single-threaded, as it stands) on the corner window of
    WINDOW cells of the headline field: assembly, then for each
    preconditioner kind its set-up and FGMRES(30) to 1e-8. Returns the
    measured times and, extrapolated to the whole grid (every cost scaled by
    the cell ratio, FGMRES by the full grid's iteration counts `its_full` when
    given, else the window's), the whole grid's solves/s."""
    import oracle as O
    from paper_1611_00127_gb300 import inputs as I
    w = I.window(p_full, *WINDOW)
    ratio = p_full.ncell / w.ncell
    u0 = I.initial_state(w)
    t0 = time.perf_counter()
    F, J, (rp, col) = O.assemble(w, u0, u0, I.DAY)
    t_asm = time.perf_counter() - t0
    parts, total_full, conv = [], t_asm * ratio, 0
    for name, kind, dec in KINDS_3D:
        t0 = time.perf_counter()
        M = O.Precond(rp, col, J, O.PrecParams(kind=kind, decouple=dec, amg=O.AmgParams(theta=THETA_3D)))
        t1 = time.perf_counter()
        x, st, its, rr = O.fgmres(rp, col, J, -F, M, m=30, rtol=1e-8, maxit=maxit)
        t2 = time.perf_counter()
        conv += int(st == 0)
        its_f = (its_full or {}).get(name, its)
        per_it = (t2 - t1) / max(its, 1)
        total_full += ratio * ((t1 - t0) + per_it * its_f)
        parts.append(f"{name}: set-up {t1 - t0:.2f} s, {its} iterations {t2 - t1:.2f} s")
    value = len(KINDS_3D) / total_full if total_full > 0 else 0.0
    return dict(value=value, unit=UNIT, cores=1, kind="oracle", extrapolated=True,
                sample=(f"window of {w.nx}x{w.ny}x{w.nz} cells of the {p_full.nx}x{p_full.ny}x{p_full.nz} field "
                        f"(1/{ratio:g} of the cells), FP64: assembly {t_asm:.2f} s; " + "; ".join(parts) +
                        f"; {conv} of {len(KINDS_3D)} converged. Extrapolated to the whole grid: every cost x "
                        f"{ratio:g} (cells), FGMRES at the whole grid's iteration counts "
                        f"{its_full if its_full else '(the window' + chr(39) + 's)'}"),
                window_conv=conv)


def host_cores():
    return os.cpu_count() or 1


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1611_00127_gb300 import inputs as I
    import oracle as O
    O.build()
    p = I.config_channel_3d(args.n3)
    vals, samples = [], []
    for w in range(args.warmup + args.steps):
        # each step: one bounded sample (the oracle on the window, extrapolated)
        r = oracle_window(p, args.maxit)
        if w >= args.warmup:
            vals.append(r["value"])
            samples.append(r["sample"])
    v = float(np.mean(vals))
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=None, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, grid=f"{args.n3}x{args.n3}x{args.n3}", solves_per_step=len(KINDS_3D),
                            gmres="FGMRES(30), rtol 1e-8, maxit %d" % args.maxit, vcycle="FP64",
                            parallelism="single host core", host_cores=host_cores()),
                cpu_baseline=dict(value=v, unit=UNIT, cores=1, kind="oracle", sample=samples[-1],
                                  extrapolated=True, host_cores=host_cores()),
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


def _oracle_member(task):
    """One ensemble member on the CPU oracle: assembly, CPR-AMG(1) set-up and
    FGMRES(30) to 1e-8 (a worker of ensemble_oracle_parallel)."""
    p, maxit = task
    import oracle as O
    from paper_1611_00127_gb300 import inputs as I
    u, uo = I.front_state(p)
    t0 = time.perf_counter()
    F, J, (rp, col) = O.assemble(p, u, uo, I.DAY)
    M = O.Precond(rp, col, J, O.PrecParams(kind=1, decouple=2))
    x, st, its, rr = O.fgmres(rp, col, J, -F, M, m=30, rtol=1e-8, maxit=maxit)
    return int(st == 0), time.perf_counter() - t0


def _ping(_):
    import oracle  # noqa: F401
    return os.getpid()


def ensemble_oracle_parallel(probs, maxit):
    """The CPU oracle (single-threaded per member, as it stands) over the
    ensemble's independent members on all host cores: a spawned process pool,
    one member per task, largest members first. Returns solves/s over the
    wall time of the whole ensemble (the pool already started)."""
    import multiprocessing as mp
    cores = host_cores()
    order = sorted(range(len(probs)), key=lambda k: -probs[k].ncell)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_ping, range(cores), chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_oracle_member, [(probs[k], maxit) for k in order], chunksize=1)
        wall = time.perf_counter() - t0
    conv = sum(r[0] for r in res)
    cpu_s = sum(r[1] for r in res)
    return dict(value=conv / wall if wall > 0 else None, unit=UNIT, cores=cores, kind="oracle", converged=conv,
                wall_s=wall, cpu_s=cpu_s,
                sample=f"all {len(probs)} members, CPR-AMG(1) FP64, assembly + set-up + FGMRES each, "
                       f"one process per host core")


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


def class_roofline(prof, peak, peak_kind, classes=None):
    """Roofline of the kernel class with the most device time in a profiled
    step: algorithmic bytes of all its launches over their summed device
    time (= bytes per launch over the average launch duration)."""
    cand = {k: v for k, v in prof.items() if v[2] > 0 and v[1] > 0 and (classes is None or k in classes)}
    if not cand:
        return None
    k = max(cand, key=lambda c: cand[c][0])
    ms, by, n = cand[k]
    achieved = by / (ms * 1e-3) / 1e9
    tr = NCU_TRAFFIC.get(k)
    return dict(bound="hbm", kernel=k, kernels=CLASS_KERNELS.get(k), achieved=achieved, peak=peak, unit="GB/s",
                frac=achieved / peak, frac_nominal=achieved / NOMINAL_HBM_GBS,
                traffic=tr[0] / n if tr else None, traffic_source=tr[1] if tr else None,
                peak_source=peak_kind, launches=n, ms=ms, bytes=by, launch_ms=ms / n, bytes_per_launch=by / n,
                how="all launches of the class in one profiled headline step: algorithmic bytes over their "
                    "summed device time (CUDA events around each call)")


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.no_extras:
        args.no_e2e = args.no_side = args.no_cpu_baseline = True
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

    from paper_1611_00127_gb300 import inputs as I
    from paper_1611_00127_gb300 import kernel_bench
    from paper_1611_00127_gb300 import rsflow as R
    R.lib()
    p = I.config_channel_3d(args.n3)
    # headline: FP32 V-cycles in FP64 FGMRES
    step = Gpu3DStep(p, R.FP32, args.maxit)
    with ClockSampler(local) as clk:
        ms32, recs32, launches = time_steps(step, args.steps, args.warmup, barrier)
    conv32 = sum(r["converged"] for r in recs32)
    # the same step with FP64 V-cycles
    k64 = min(args.steps, 3)
    ms64, recs64, conv64 = 0.0, [], 0
    if not args.no_extras:
        step64 = Gpu3DStep(p, R.FP64, args.maxit)
        ms64, recs64, _ = time_steps(step64, k64, 1, barrier)
        conv64 = sum(r["converged"] for r in recs64)
        del step64
    # end to end: the same step from pinned host buffers
    e2e = None
    te_ms, ce, ke = 0.0, 0, min(args.steps, 5)
    if not args.no_e2e:
        host = dict(k=torch.from_numpy(np.ascontiguousarray(np.stack([p.kx, p.ky, p.kz]))).pin_memory(),
                    u=torch.from_numpy(I.initial_state(p)).pin_memory())
        stepe = Gpu3DStep(p, R.FP32, args.maxit, host=host)
        ce, te_s = e2e_wall(stepe, ke, 1)
        te_ms = te_s * 1e3
        h2d, d2h = stepe.h2d, stepe.d2h
        del stepe, host
    (ms32, ms64, te_ms), (conv32, conv64, ce) = reduce_over_ranks([ms32, ms64, te_ms], [conv32, conv64, ce],
                                                                  dist, "cuda")
    # (every step solves the same systems: the last step's converged count holds for each)
    value = solves_per_second(conv32, args.steps, ms32)
    value64 = solves_per_second(conv64, k64, ms64)
    if not args.no_e2e:
        e2e = dict(value=solves_per_second(ce, 1, te_ms), unit=UNIT, h2d_bytes_per_step=h2d,
                   d2h_bytes_per_step=d2h, steps=ke,
                   how="public API, permeability and state copied in from pinned host memory and both "
                       "solutions copied out inside every step, wall clock")
    if rank != 0:
        return
    if args.no_extras:
        print(json.dumps(dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                              warmup=args.warmup, ms_per_step=ms32 / args.steps, higher_is_better=True,
                              scaling="weak", vs_baseline=None, dtype="f64+f32", data="synthetic",
                              config=dict(workload=WORKLOAD, grid=f"{args.n3}x{args.n3}x{args.n3}",
                                          note="headline timing only (--no-extras)"),
                              solves=recs32, gpu_launches=int(launches))))
        return
    peak, peak_kind = hbm_peak()
    # per kernel class, one profiled headline step
    prof, per_solve = profiled_step(step)
    hier = dict(getattr(step, "hier", {}))
    roofline = class_roofline(prof, peak, peak_kind)
    roofline_solve = class_roofline(prof, peak, peak_kind,
                                    classes=("hybrid_gs_sweep", "csr_resid_restrict_prolong", "bsr2_spmv",
                                             "gmres_cgs2"))
    kernel_profile = {k: dict(ms=v[0], gbs=(v[1] / (v[0] * 1e-3) / 1e9 if v[0] > 0 else 0.0), launches=v[2])
                      for k, v in prof.items() if v[2] > 0}
    del step
    torch.cuda.empty_cache()
    # level-0 kernels of the headline's CPR hierarchy, L2 flushed, both precisions
    level0 = {}
    for pname, prec in (("fp32", R.FP32), ("fp64", R.FP64)):
        k = kernel_bench.channel(args.n3, prec, R.CPR1, reps=20, p=p)
        sw = k["sweep_bytes"] / (k["sweep_ms"] * 1e-3) / 1e9
        sp = k["spmv_bytes"] / (k["spmv_ms"] * 1e-3) / 1e9
        level0[pname] = dict(
            rows=k["rows"], nnz=k["nnz"],
            k_hgs=dict(launch_ms=k["sweep_ms"], bytes_per_launch=k["sweep_bytes"], achieved=sw, frac=sw / peak,
                       frac_nominal=sw / NOMINAL_HBM_GBS),
            k_bsr2_spmv=dict(launch_ms=k["spmv_ms"], bytes_per_launch=k["spmv_bytes"], achieved=sp, frac=sp / peak,
                             frac_nominal=sp / NOMINAL_HBM_GBS, nnzb=k["nnzb"]),
            transfer={t: dict(launch_ms=v["ms"], bytes_per_launch=v["bytes"], achieved=v["gbs"],
                              frac=v["gbs"] / peak, frac_nominal=v["gbs"] / NOMINAL_HBM_GBS)
                      for t, v in k["transfer"].items()})
        torch.cuda.empty_cache()
    side = {}
    if not args.no_side:
        # 128^3 layered grid, FP32 and FP64 V-cycles
        p128 = I.config_layered_3d(128)
        for pname, prec in (("fp32", R.FP32), ("fp64", R.FP64)):
            st = Gpu3DStep(p128, prec, args.maxit)
            m, r, _ = time_steps(st, 3, 1, barrier)
            side[f"layered128_{pname}"] = dict(value=solves_per_second(sum(x["converged"] for x in r), 3, m),
                                               ms_per_step=m / 3, solves=r)
            del st
        side["layered128_fp32_over_fp64"] = (side["layered128_fp32"]["value"] / side["layered128_fp64"]["value"]
                                             if side["layered128_fp64"]["value"] else None)
        torch.cuda.empty_cache()
        # 256x256 log-normal grid: 12 solves per step
        probs, states = workload(args.n)
        for pname, prec, cls in (("fp64", R.FP64, GpuStep), ("fp32", R.FP32, GpuStep),
                                 ("fp32_batched", R.FP32, GpuBatchStep)):
            st = cls(probs, states, prec, args.maxit)
            m, r, _ = time_steps(st, 3, 1, barrier)
            side[f"lognormal256_{pname}"] = dict(value=solves_per_second(sum(x["converged"] for x in r), 3, m),
                                                 ms_per_step=m / 3, converged_per_step=sum(x["converged"] for x in r),
                                                 solves=r)
            del st
        side["lognormal256_workload"] = WORKLOAD_2D
        side["lognormal256_bf_restriction"] = "lAIR (localised approximate ideal restriction)"
        torch.cuda.empty_cache()
    ensemble = None
    if not (args.no_ensemble or args.no_side):
        ensemble = ensemble_bench(600)
        if not args.no_cpu_baseline:
            from paper_1611_00127_gb300 import inputs as I2
            ensemble["cpu_oracle_parallel"] = ensemble_oracle_parallel(I2.config_ensemble(), 600)
    newton = newton_sequence(p, args.maxit) if args.newton else None
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_window(p, args.maxit, its_full={r["prec"]: r["its"] for r in recs32})
        cpu["host_cores"] = host_cores()
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms32 / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64+f32",
        data="synthetic",
        config=dict(workload=WORKLOAD, grid=f"{args.n3}x{args.n3}x{args.n3}", dof=2 * p.ncell,
                    preconditioners=["CPR-AMG(1), quasi-IMPES, point-block Jacobi P1",
                                     "block factorisation, SIMPLE Schur complement"],
                    solves_per_step=len(KINDS_3D), converged_per_step=conv32 // max(world, 1),
                    gmres="FP64 FGMRES(30), rtol 1e-8, maxit %d" % args.maxit, vcycle="FP32",
                    amg="PMIS, ext+i, theta 0.5, hybrid multicolour Gauss-Seidel V(1,1)",
                    l2="flushed (256 MB write) before every timed step; working set > L2",
                    parallelism="replicas" if world > 1 else "single GPU"),
        solves=recs32,
        fp64_vcycle=dict(value=value64, ms_per_step=ms64 / k64, steps=k64, solves=recs64,
                         fp32_over_fp64=value / value64 if value64 > 0 else None),
        clocks=clk.summary(),
        roofline=roofline,
        roofline_solve=roofline_solve,
        level0_kernels=level0,
        kernel_profile=dict(note="one eager profiled headline step, CUDA events per launch", classes=kernel_profile),
        hierarchies=hier,
        side=side,
        ensemble=ensemble,
        newton=newton,
        gpu_launches=int(launches),
        e2e=e2e,
        cpu_baseline=cpu,
    )
    print(json.dumps(line))


def newton_sequence(p, maxit, steps=5):
    """The headline grid's full Newton sequence: `steps` one-day backward-Euler
    steps from the initial state, with CPR-AMG and with block factorisation
    (FP32 V-cycles). Each Newton iteration is one Jacobian solve; solves/s is
    Newton iterations over the wall time of the sequence."""
    import torch
    from paper_1611_00127_gb300 import inputs as I
    from paper_1611_00127_gb300 import rsflow as R
    dp = R.DeviceProblems(p)
    out = {}
    for name, kind, dec in KINDS_3D:
        prm = R.NewtonParams(prec=R.PrecParams(kind=kind, decouple=dec,
                                               amg=R.AmgParams(theta=THETA_3D, precision=R.FP32)),
                             gmres=R.GmresParams(maxit=maxit))
        u = torch.as_tensor(I.initial_state(p), device="cuda")
        per, nits, t0 = [], 0, time.perf_counter()
        for k in range(steps):
            u_old = u.clone()
            rc, st = R.newton_step(dp, u, u_old, I.DAY, prm)
            nits += st["newton_its"]
            per.append(dict(step=k, rc=rc, **st))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[name] = dict(steps=per, newton_its=nits, wall_s=wall, solves_per_s=nits / wall if wall > 0 else None)
    return out


if __name__ == "__main__":
    main()

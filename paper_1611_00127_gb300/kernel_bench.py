"""Kernel microbenchmark: the hybrid Gauss-Seidel sweep of AMG level 0 and the
block SpMV, timed back to back with CUDA events on the launching stream.

    python -m paper_1611_00127_gb300.kernel_bench [--grid layered3d|channel3d|lognormal2d]
        [--n N] [--pc PC] [--prec fp64|fp32] [--reps 20] [--kind cpr1|bf] [--ilu]

The case is the exact Newton Jacobian at the synthetic front state of the
n^3 layered log-normal grid (7-point two-point-flux stencil of Sec. 2 in 3D;
L2 flushed before each timed loop, the working set exceeds L2) or of the
n x n log-normal grid with capillary scale PC (operands L2-resident, as in
a solve of that size). Level 0 is the pressure block A_pp of the
quasi-IMPES-decoupled Jacobian (CPR, Alg. 1) or the SIMPLE Schur complement
(block factorisation, Alg. 3). Each loop sits in an NVTX
range ("sweep", "spmv"), so a profiler can select exactly those launches.
Prints one JSON object: per-launch time and algorithmic bytes of each kernel.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import inputs as I
from . import rsflow as R


def bsr2_spmv_bytes(J: R.Bsr2) -> float:
    """Algorithmic bytes of one y = J x: every block (32 B) and column index
    (4 B) once, the row pointers, x and y once each (16 B per cell)."""
    return J.nnzb * 36.0 + (J.nb + 1) * 4.0 + J.nb * 32.0


class Level0Case:
    """Assembled Jacobian, preconditioner and level-0 hierarchy of one grid."""

    def __init__(self, p, state, precision: int, kind: int = R.CPR1, theta: float = 0.5, chunk: int = 512):
        self.p = p
        self.precision = precision
        u, uo = state
        self.dp = R.DeviceProblems(p)
        self.J = R.Bsr2.pattern(self.dp)
        self.F = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
        R.jacobian_assemble(self.dp, torch.as_tensor(u, device="cuda"), torch.as_tensor(uo, device="cuda"),
                            I.DAY, self.J, self.F)
        self.M = R.Precond(self.J, R.PrecParams(kind=kind, amg=R.AmgParams(theta=theta, precision=precision,
                                                                           chunk=chunk)))
        self.H = self.M.amg(0)
        z = torch.empty_like(self.F)
        self.M.apply(self.F, z)          # leaves a right-hand side on every level
        self.y = torch.empty_like(self.F)
        self.lanes = R.autotune_bsr2(self.J, self.F, self.y)     # lanes per block row of the SpMV

    def time_sweeps(self, reps: int, flush: torch.Tensor | None = None):
        """(ms per sweep, algorithmic bytes per sweep) over `reps` back-to-back
        level-0 sweeps."""
        self.H.level_smooth(0, 3)
        if flush is not None:
            flush.add_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("sweep")
        e0.record()
        by = self.H.level_smooth(0, reps)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return e0.elapsed_time(e1) / reps, by

    def time_spmv(self, reps: int, flush: torch.Tensor | None = None):
        """(ms per launch, algorithmic bytes per launch) of y = J x."""
        for _ in range(3):
            R.bsr2_spmv(self.J, self.F, self.y)
        if flush is not None:
            flush.add_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("spmv")
        e0.record()
        for _ in range(reps):
            R.bsr2_spmv(self.J, self.F, self.y)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return e0.elapsed_time(e1) / reps, bsr2_spmv_bytes(self.J)

    def time_transfer(self, which: int, reps: int, flush: torch.Tensor | None = None):
        """(ms per launch, algorithmic bytes per launch) of one level-0
        transfer kernel: 0 residual, 1 restriction, 2 prolongation."""
        self.H.level_transfer(0, which, 3)
        if flush is not None:
            flush.add_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(("residual", "restrict", "prolong")[which])
        e0.record()
        by = self.H.level_transfer(0, which, reps)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return e0.elapsed_time(e1) / reps, by

    def time_ilu(self, reps: int):
        """(ms per apply, levels, widest level) of the ILU(0) triangular solves
        on J (the first stage of CPR with P1 = ILU(0)) in the case's
        precision."""
        f = R.Ilu0(self.J, self.precision)
        y = torch.empty_like(self.F)
        for _ in range(3):
            f.apply(self.F, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("ilu")
        e0.record()
        for _ in range(reps):
            f.apply(self.F, y)
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        nlev, maxw, _ = f.info()
        f.close()
        return e0.elapsed_time(e1) / reps, nlev, maxw

    def level0(self):
        n0, nnz0 = self.H.level_info(0)[:2]
        return n0, nnz0

    def close(self):
        self.M.close()


def layered(n: int, precision: int, kind: int = R.CPR1, reps: int = 20, chunk: int = 512) -> dict:
    """Sweep and SpMV timings on the n^3 layered workload, L2 flushed."""
    p = I.config_layered_3d(n)
    case = Level0Case(p, I.front_state(p), precision, kind, chunk=chunk)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    ts, bs = case.time_sweeps(reps, flush)
    tm, bm = case.time_spmv(reps, flush)
    xfer = {}
    for which, name in enumerate(("residual", "restrict", "prolong")):
        t, by = case.time_transfer(which, reps, flush)
        xfer[name] = dict(ms=t, bytes=by, gbs=by / (t * 1e-3) / 1e9)
    n0, nnz0 = case.level0()
    nnzb = case.J.nnzb
    case.close()
    return dict(sweep_ms=ts, sweep_bytes=bs, rows=n0, nnz=nnz0, spmv_ms=tm, spmv_bytes=bm, nnzb=nnzb,
                spmv_lanes=case.lanes, transfer=xfer)


def channel(n: int, precision: int, kind: int = R.CPR1, reps: int = 20, chunk: int = 512, p=None) -> dict:
    """Sweep, transfer and SpMV timings on the n^3 channelised workload at
    its first Newton Jacobian (u = u_old = the initial state), L2 flushed."""
    p = p if p is not None else I.config_channel_3d(n)
    u0 = I.initial_state(p)
    case = Level0Case(p, (u0, u0), precision, kind, chunk=chunk)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    ts, bs = case.time_sweeps(reps, flush)
    tm, bm = case.time_spmv(reps, flush)
    xfer = {}
    for which, name in enumerate(("residual", "restrict", "prolong")):
        t, by = case.time_transfer(which, reps, flush)
        xfer[name] = dict(ms=t, bytes=by, gbs=by / (t * 1e-3) / 1e9)
    n0, nnz0 = case.level0()
    nnzb = case.J.nnzb
    case.close()
    return dict(sweep_ms=ts, sweep_bytes=bs, rows=n0, nnz=nnz0, spmv_ms=tm, spmv_bytes=bm, nnzb=nnzb,
                spmv_lanes=case.lanes, transfer=xfer)


def lognormal(n: int, pc: float, precision: int, kind: int = R.BF, reps: int = 50, flush_l2: bool = False,
              chunk: int = 512) -> dict:
    """Sweep and SpMV timings on the n x n log-normal grid with capillary scale
    `pc` (2D strength threshold 0.25). Without `flush_l2` the operands stay
    in L2 between launches, as they do inside a solve of this size."""
    p = I.config_lognormal_2d(pc, n=n)
    case = Level0Case(p, I.front_state(p), precision, kind, theta=0.25, chunk=chunk)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda") if flush_l2 else None
    ts, bs = case.time_sweeps(reps, flush)
    tm, bm = case.time_spmv(reps, flush)
    n0, nnz0 = case.level0()
    nnzb = case.J.nnzb
    case.close()
    return dict(sweep_ms=ts, sweep_bytes=bs, rows=n0, nnz=nnz0, spmv_ms=tm, spmv_bytes=bm, nnzb=nnzb,
                spmv_lanes=case.lanes)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", choices=["layered3d", "channel3d", "lognormal2d"], default="layered3d")
    ap.add_argument("--n", type=int, default=None, help="cells per side (128 for 3D, 256 for 2D)")
    ap.add_argument("--pc", type=float, default=1e3, help="capillary scale of the 2D grid")
    ap.add_argument("--prec", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--kind", choices=["cpr1", "bf"], default="cpr1")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--chunk", type=int, default=512, help="rows per chunk of the hybrid smoother")
    ap.add_argument("--ilu", action="store_true", help="time the ILU(0) solves on J instead")
    a = ap.parse_args()
    prec = R.FP64 if a.prec == "fp64" else R.FP32
    kind = R.CPR1 if a.kind == "cpr1" else R.BF
    if a.ilu:
        a.n = a.n or (128 if a.grid == "layered3d" else 256)
        p = I.config_layered_3d(a.n) if a.grid == "layered3d" else I.config_lognormal_2d(a.pc, n=a.n)
        case = Level0Case(p, I.front_state(p), prec, kind)
        ms, nlev, maxw = case.time_ilu(a.reps)
        case.close()
        print(json.dumps(dict(grid=a.grid, n=a.n, prec=a.prec, ilu_ms=ms, levels=nlev, widest=maxw,
                              us_per_level_step=1e3 * ms / (2 * nlev))))
        return
    if a.grid == "layered3d":
        a.n = a.n or 128
        r = layered(a.n, prec, kind, a.reps, a.chunk)
    elif a.grid == "channel3d":
        a.n = a.n or 256
        r = channel(a.n, prec, kind, a.reps, a.chunk)
    else:
        a.n = a.n or 256
        r = lognormal(a.n, a.pc, prec, kind, a.reps, chunk=a.chunk)
    r.update(grid=a.grid, n=a.n, prec=a.prec, kind=a.kind, chunk=a.chunk,
             sweep_gbs=r["sweep_bytes"] / (r["sweep_ms"] * 1e-3) / 1e9,
             spmv_gbs=r["spmv_bytes"] / (r["spmv_ms"] * 1e-3) / 1e9,
             device_used_gb=(lambda fr: (fr[1] - fr[0]) / 1e9)(torch.cuda.mem_get_info()))
    print(json.dumps(r))


if __name__ == "__main__":
    main()

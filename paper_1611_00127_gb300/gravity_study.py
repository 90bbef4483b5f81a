"""Gravity-driven two-dimensional study (Sec. 4.2, Tables 2d_grav_diff,
2d_grav_adv and 2d_grav_hyp) run through the C-ABI on the GPU.

A vertical 20 m x 20 m box of 100 mD on meshes 20^2 .. 160^2, water injected
at 5 m^3/day into the top-left cell, outlet at the top-right cell, the
capillary parameter sets Ex 1 (diffusion-dominated, dt = 10 days), Ex 2
(advection-dominated, dt = 4 days) and Ex 3 (strongly advection-dominated,
dt = 1 day), two backward-Euler steps each (final times 20, 8 and 2 days).
Every step is Newton's method (`newton_step`) with one of the preconditioners
inside FGMRES; the study reports the Newton iterations (NI), the linear
iterations (LI) and LI/NI per mesh, the quantity the tables print, and so
checks how each preconditioner's iteration count depends on the mesh size.

    python -m paper_1611_00127_gb300.gravity_study [--meshes 20 40 80 160]
        [--examples 1 2 3] [--kinds AMG CPR1 CPR2 BF] [--pc bc|linear]
        [--prec fp64|fp32] [--rtol 1e-8] [--json out.json]

Newton takes full steps except that each cell's S_n change is cut to
[-0.2, 0.2] per iteration (an Appleyard chop): from the uniform initial state
the first undamped Newton updates of this problem move the water pressure by
~1e8 Pa, drive S_n to both bounds and leave a singular Jacobian. The paper
does not state its damping.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import inputs as I
from . import rsflow as R

# preconditioner name -> (kind, decoupling, P1); CPR uses the quasi-IMPES
# decoupling with P1 = ILU(0) (the paper's choice) or point-block Jacobi,
# AMG is the systems (point) AMG on the whole Jacobian
KINDS = {
    "AMG": (R.AMG_J, R.DECOUPLE_NONE, R.P1_BLOCK_JACOBI),
    "CPR1": (R.CPR1, R.DECOUPLE_QIMPES, R.P1_ILU0),
    "CPR2": (R.CPR2, R.DECOUPLE_QIMPES, R.P1_ILU0),
    "BF": (R.BF, R.DECOUPLE_NONE, R.P1_BLOCK_JACOBI),
    "CPR1_BJ": (R.CPR1, R.DECOUPLE_QIMPES, R.P1_BLOCK_JACOBI),
    "CPR2_BJ": (R.CPR2, R.DECOUPLE_QIMPES, R.P1_BLOCK_JACOBI),
    "AMG_SCALAR": (R.AMG_J_SCALAR, R.DECOUPLE_NONE, R.P1_BLOCK_JACOBI),
}
MESHES = (20, 40, 80, 160)
MAX_DS = 0.2


def newton_params(kind: str, precision: int = R.FP64, rtol: float = 1e-8, max_newton: int = 40,
                  max_ds: float = MAX_DS) -> R.NewtonParams:
    k, dec, p1 = KINDS[kind]
    return R.NewtonParams(max_newton=max_newton, ftol=1e-6, max_ds=max_ds,
                          gmres=R.GmresParams(m=30, maxit=1000, rtol=rtol),
                          prec=R.PrecParams(kind=k, decouple=dec, p1=p1, amg=R.AmgParams(precision=precision)))


def run_case(n: int, example: int, kind: str, pc_model: int = I.PC_BROOKS_COREY, precision: int = R.FP64,
             rtol: float = 1e-8, steps: int = I.GRAVITY_STEPS, keep_states: bool = False) -> dict:
    """Time-step the n x n gravity box with Newton + FGMRES preconditioned by
    `kind`. Returns per-step and total NI/LI, whether every step converged
    (a step that does not ends the run), wall time, and optionally the state
    after each step (host arrays)."""
    p = I.config_gravity_2d(n, example, pc_model)
    dt = I.GRAVITY_DT_DAYS[example] * I.DAY
    dp = R.DeviceProblems(p)
    prm = newton_params(kind, precision, rtol)
    u = torch.as_tensor(I.uniform_state(p), device="cuda")
    out = dict(n=n, example=example, kind=kind, pc_model=pc_model, dt_days=dt / I.DAY, steps=[], converged=True)
    states = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        u_old = u.clone()
        rc, st = R.newton_step(dp, u, u_old, dt, prm)
        out["steps"].append(dict(ni=st["newton_its"], li=st["linear_its"], fnorm=st["fnorm"], status=rc))
        if rc != R.RS_OK:
            out["converged"] = False
            break
        if keep_states:
            states.append(u.cpu().numpy())
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    out["NI"] = sum(s["ni"] for s in out["steps"])
    out["LI"] = sum(s["li"] for s in out["steps"])
    out["LI_per_NI"] = out["LI"] / max(out["NI"], 1)
    if keep_states:
        out["states"] = states
    return out


def table(results: list, example: int, kinds, meshes) -> str:
    """LI/NI per preconditioner and mesh in the layout of the paper's tables
    ('-' where a step did not converge)."""
    by = {(r["kind"], r["n"]): r for r in results if r["example"] == example}
    head = f"Ex {example} (dt = {I.GRAVITY_DT_DAYS[example]:g} days)  " + "  ".join(f"{m}^2".rjust(7) for m in meshes)
    lines = [head]
    for k in kinds:
        cells = []
        for m in meshes:
            r = by.get((k, m))
            cells.append("      -" if r is None or not r["converged"] else f"{r['LI_per_NI']:7.1f}")
        lines.append(f"{k:<28s}" + "  ".join(cells))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--meshes", type=int, nargs="+", default=list(MESHES))
    ap.add_argument("--examples", type=int, nargs="+", default=[1, 2, 3])
    ap.add_argument("--kinds", nargs="+", default=["AMG", "CPR1", "CPR2", "BF"], choices=list(KINDS))
    ap.add_argument("--pc", choices=["bc", "linear"], default="bc")
    ap.add_argument("--prec", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--json", default=None, help="write every result to this file")
    a = ap.parse_args()
    pcm = I.PC_BROOKS_COREY if a.pc == "bc" else I.PC_LINEAR
    prec = R.FP64 if a.prec == "fp64" else R.FP32
    R.lib()
    results = []
    for ex in a.examples:
        for k in a.kinds:
            for m in a.meshes:
                r = run_case(m, ex, k, pcm, prec, a.rtol)
                results.append(r)
                print(json.dumps({key: v for key, v in r.items() if key != "states"}), flush=True)
    for ex in a.examples:
        print(table(results, ex, a.kinds, a.meshes))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(results, f, indent=1)


if __name__ == "__main__":
    main()

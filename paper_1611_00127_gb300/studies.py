"""Newton time-stepping studies of Sec. 4 run through the C-ABI on the GPU,
reporting the Newton iterations (NI), the linear iterations (LI) and LI/NI
per preconditioner, the quantities the paper's tables print.

* gravity: the gravity-driven two-dimensional study (Sec. 4.2, Tables
  2d_grav_diff, 2d_grav_adv, 2d_grav_hyp). A vertical 20 m x 20 m box of
  100 mD on meshes 20^2 .. 160^2, water injected at 5 m^3/day into the
  top-left cell, outlet at the top-right cell, capillary parameter sets Ex 1
  (diffusion-dominated, dt = 10 days), Ex 2 (advection-dominated, dt = 4
  days) and Ex 3 (strongly advection-dominated, dt = 1 day), two steps each
  (final times 20, 8 and 2 days). Checks how each preconditioner's
  iteration count depends on the mesh size.
* oil-water: the two-dimensional oil-water example of Sec. 4.1 (Tables
  performance_q5_1 .. q5_3) on a seeded stand-in for its SPE10 section:
  100 x 20 cells over 762 m x 15.24 m, 50 m^3/day injected at the lower-left
  corner, outlet at the top right, 200 days in steps of 20 days, the linear
  and the Brooks-Corey capillary model with parameter sets Ex 1 .. Ex 4.

    python -m paper_1611_00127_gb300.studies gravity [--meshes 20 40 80 160]
        [--examples 1 2 3] [--kinds AMG CPR1 CPR2 BF] [--pc bc|linear]
        [--prec fp64|fp32] [--rtol 1e-8] [--restriction 0|1|3] [--json out.json]
    python -m paper_1611_00127_gb300.studies oil-water [--examples 1 2 3 4]
        [--pc linear bc] [--kinds ...] [--prec ...] [--rtol ...] [--restriction ...]
        [--json ...]

Newton takes full steps except that each cell's S_n change is cut to
[-0.2, 0.2] per iteration (an Appleyard chop): from the uniform initial state
the first undamped Newton updates of the gravity box move the water pressure
by ~1e8 Pa, drive S_n to both bounds and leave a singular Jacobian. The paper
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
                  max_ds: float = MAX_DS, restriction: int = 0) -> R.NewtonParams:
    k, dec, p1 = KINDS[kind]
    return R.NewtonParams(max_newton=max_newton, ftol=1e-6, max_ds=max_ds,
                          gmres=R.GmresParams(m=30, maxit=1000, rtol=rtol),
                          prec=R.PrecParams(kind=k, decouple=dec, p1=p1,
                                            amg=R.AmgParams(precision=precision, restriction=restriction)))


def run_steps(p, dt: float, steps: int, kind: str, precision: int = R.FP64, rtol: float = 1e-8,
              keep_states: bool = False, restriction: int = 0) -> dict:
    """Time-step grid `p` from the uniform initial state (p_w = 1e5 Pa,
    S_n = 0.8) with Newton + FGMRES preconditioned by `kind`. Returns per-step
    and total NI/LI, whether every step converged (a step that does not ends
    the run), wall time, and optionally the state after each step (host
    arrays). `restriction` is the scalar hierarchies' restriction (0 Galerkin,
    the paper's; 1 AIR; 3 lAIR)."""
    dp = R.DeviceProblems(p)
    prm = newton_params(kind, precision, rtol, restriction=restriction)
    u = torch.as_tensor(I.uniform_state(p), device="cuda")
    out = dict(kind=kind, pc_model=p.pc_model, dt_days=dt / I.DAY, steps=[], converged=True)
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


def run_case(n: int, example: int, kind: str, pc_model: int = I.PC_BROOKS_COREY, precision: int = R.FP64,
             rtol: float = 1e-8, steps: int = I.GRAVITY_STEPS, keep_states: bool = False,
             restriction: int = 0) -> dict:
    """One (mesh, example, preconditioner) case of the gravity study."""
    p = I.config_gravity_2d(n, example, pc_model)
    out = run_steps(p, I.GRAVITY_DT_DAYS[example] * I.DAY, steps, kind, precision, rtol, keep_states, restriction)
    out.update(n=n, example=example)
    return out


def run_oil_water(example: int, pc_model: int, kind: str, precision: int = R.FP64, rtol: float = 1e-8,
                  steps: int = I.OIL_WATER_STEPS, keep_states: bool = False, restriction: int = 0) -> dict:
    """One (example, capillary model, preconditioner) case of the oil-water
    study."""
    p = I.config_oil_water_2d(example, pc_model)
    out = run_steps(p, I.OIL_WATER_DT_DAYS * I.DAY, steps, kind, precision, rtol, keep_states, restriction)
    out.update(example=example)
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


def oil_water_table(results: list, kinds, examples, models) -> str:
    """NI, LI and LI/NI per preconditioner, example and capillary model."""
    lines = []
    for ex in examples:
        lines.append(f"Ex {ex}" + "".join(f"   {('linear' if m == I.PC_LINEAR else 'Brooks-Corey'):>22s}"
                                           for m in models))
        for k in kinds:
            cells = []
            for m in models:
                r = next((r for r in results if r["example"] == ex and r["kind"] == k and r["pc_model"] == m), None)
                cells.append(f"   {'-':>22s}" if r is None or not r["converged"] else
                             f"   {r['NI']:5d} {r['LI']:6d} {r['LI_per_NI']:9.1f}")
            lines.append(f"{k:<12s}" + "".join(cells))
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["gravity", "oil-water"])
    ap.add_argument("--meshes", type=int, nargs="+", default=list(MESHES))
    ap.add_argument("--examples", type=int, nargs="+", default=None)
    ap.add_argument("--kinds", nargs="+", default=["AMG", "CPR1", "CPR2", "BF"], choices=list(KINDS))
    ap.add_argument("--pc", nargs="+", choices=["bc", "linear"], default=None)
    ap.add_argument("--prec", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--restriction", type=int, choices=[0, 1, 3], default=0,
                    help="scalar AMG restriction: 0 Galerkin (the paper's), 1 AIR, 3 lAIR")
    ap.add_argument("--json", default=None, help="write every result to this file")
    a = ap.parse_args()
    prec = R.FP64 if a.prec == "fp64" else R.FP32
    R.lib()
    results = []
    if a.study == "gravity":
        pcm = I.PC_BROOKS_COREY if (a.pc or ["bc"])[0] == "bc" else I.PC_LINEAR
        examples = a.examples or [1, 2, 3]
        for ex in examples:
            for k in a.kinds:
                for m in a.meshes:
                    r = run_case(m, ex, k, pcm, prec, a.rtol, restriction=a.restriction)
                    results.append(r)
                    print(json.dumps(r), flush=True)
        for ex in examples:
            print(table(results, ex, a.kinds, a.meshes))
    else:
        models = [I.PC_BROOKS_COREY if m == "bc" else I.PC_LINEAR for m in (a.pc or ["linear", "bc"])]
        examples = a.examples or [1, 2, 3, 4]
        for ex in examples:
            for m in models:
                for k in a.kinds:
                    r = run_oil_water(ex, m, k, prec, a.rtol, restriction=a.restriction)
                    results.append(r)
                    print(json.dumps(r), flush=True)
        print(oil_water_table(results, a.kinds, examples, models))
    if a.json:
        with open(a.json, "w") as f:
            json.dump(results, f, indent=1)


if __name__ == "__main__":
    main()

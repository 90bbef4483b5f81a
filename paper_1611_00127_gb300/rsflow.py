"""Thin Python binding of the rsflow C-ABI (``include/rsflow.h``).

Argument marshalling only: every step of the solver runs in the CUDA library.
PyTorch supplies device memory (tensors) and the current CUDA stream. The
library must be built (``paper_1611_00127_gb300.build``); importing this
module on a machine without it raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

RS_OK, RS_NOT_CONVERGED = 0, 1
RS_EINVAL, RS_ECUDA, RS_ETIMEOUT = -1, -2, -3
AMG_J, CPR1, CPR2, BF, AMG_J_SCALAR = 0, 1, 2, 3, 4
DECOUPLE_NONE, DECOUPLE_ABF, DECOUPLE_QIMPES = 0, 1, 2
P1_BLOCK_JACOBI, P1_ILU0 = 0, 1
FP32, FP64 = 0, 1

_lib = None


class RsError(RuntimeError):
    pass


def lib():
    """Load the CUDA library, building it first when nvcc is available."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not _build.up_to_date():
            try:
                path = _build.build()
            except Exception as e:  # no toolchain: the library must already exist
                if not os.path.exists(path):
                    raise RsError(f"rsflow CUDA library missing and cannot be built: {e}") from e
        L = C.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("kx", C.c_void_p), ("ky", C.c_void_p), ("kz", C.c_void_p),
                ("phi", C.c_double), ("mu_w", C.c_double), ("mu_n", C.c_double),
                ("rho_w", C.c_double), ("rho_n", C.c_double), ("g", C.c_double),
                ("pc_model", C.c_int32), ("pc_p0", C.c_double), ("pc_pd", C.c_double),
                ("bc_lambda", C.c_double), ("s_wr", C.c_double), ("s_nr", C.c_double),
                ("u_in", C.c_double), ("p_out", C.c_double), ("sn_out", C.c_double),
                ("q_in", C.c_double), ("well_in", C.c_int32), ("well_out", C.c_int32)]


class Bsr2C(C.Structure):
    _fields_ = [("nb", C.c_int32), ("nnzb", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("nseg", C.c_int32), ("seg_off", C.c_void_p)]


class CsrC(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("nseg", C.c_int32), ("seg_off", C.c_void_p)]


class AmgParamsC(C.Structure):
    _fields_ = [("theta", C.c_double), ("seed", C.c_uint64), ("max_levels", C.c_int32),
                ("coarse_n", C.c_int32), ("max_dense", C.c_int32), ("smoother", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("interp", C.c_int32),
                ("num_functions", C.c_int32), ("precision", C.c_int32), ("chunk", C.c_int32),
                ("agg_levels", C.c_int32), ("chunk_coarse", C.c_int32),
                ("restriction", C.c_int32)]


class PrecParamsC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("decouple", C.c_int32), ("p1", C.c_int32), ("amg", AmgParamsC)]


class GmresParamsC(C.Structure):
    _fields_ = [("m", C.c_int32), ("maxit", C.c_int32), ("rtol", C.c_double)]


class GmresStatsC(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("relres", C.c_double),
                ("its", C.c_void_p), ("relres_seg", C.c_void_p)]


class NewtonParamsC(C.Structure):
    _fields_ = [("max_newton", C.c_int32), ("ftol", C.c_double), ("gmres", GmresParamsC),
                ("prec", PrecParamsC), ("max_ds", C.c_double)]


class NewtonStatsC(C.Structure):
    _fields_ = [("newton_its", C.c_int32), ("linear_its", C.c_int32), ("fnorm", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("assemble_ms", C.c_double)]


def _declare(L):
    P, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "rs_last_error": (C.c_char_p, []),
        "rs_version": (C.c_int, [P, P, P]),
        "rs_bsr2_nnzb": (i64, [P, i32]),
        "rs_bsr2_pattern": (C.c_int, [P, i32, P, P, P]),
        "jacobian_assemble": (C.c_int, [P, i32, P, P, f64, P, P, P]),
        "jacobian_assemble_noalloc": (C.c_int, [P, i32, P, P, f64, P, P, P]),
        "amg_setup": (C.c_int, [P, P, P, P]),
        "amg_destroy": (C.c_int, [P]),
        "amg_apply": (C.c_int, [P, P, P, P]),
        "amg_levels": (C.c_int, [P, P]),
        "amg_level_info": (C.c_int, [P, i32, P, P, P, P]),
        "amg_level_copy": (C.c_int, [P, i32, P, P, P, P, P, P, P, P, P]),
        "amg_level_smooth": (C.c_int, [P, i32, i32, P, P]),
        "amg_level_transfer": (C.c_int, [P, i32, i32, i32, P, P]),
        "ilu0_create": (C.c_int, [P, i32, P, P]),
        "ilu0_apply": (C.c_int, [P, P, P, P]),
        "ilu0_info": (C.c_int, [P, P, P, P]),
        "ilu0_factors": (C.c_int, [P, P, P]),
        "ilu0_destroy": (C.c_int, [P]),
        "precond_create": (C.c_int, [P, P, P, P]),
        "precond_destroy": (C.c_int, [P]),
        "precond_apply": (C.c_int, [P, P, P, P]),
        "precond_amg": (P, [P, i32]),
        "gmres_solve": (C.c_int, [P, P, P, P, P, P, P]),
        "newton_step": (C.c_int, [P, i32, P, P, f64, P, P, P]),
        "bsr2_spmv": (C.c_int, [P, P, P, P]),
        "bsr2_residual": (C.c_int, [P, P, P, P, P]),
        "rs_tune_set_bsr2_lpr": (C.c_int, [C.c_int]),
        "rs_autotune_bsr2": (C.c_int, [P, P, P, P, P]),
        "rs_launch_count": (C.c_longlong, []),
        "rs_wait_status": (C.c_int, [P]),
        "rs_raise_wait_flag": (C.c_int, [P]),
        "rs_profile_begin": (C.c_int, []),
        "rs_profile_end": (C.c_int, [P, P, P, C.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise RsError(f"{what} failed ({rc}): {lib().rs_last_error().decode()}")
    return rc


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ problems
class DeviceProblems:
    """Grids of one batch with their permeability fields on the device."""

    def __init__(self, probs, device="cuda"):
        if not isinstance(probs, (list, tuple)):
            probs = [probs]
        self.probs = list(probs)
        self._keep = []
        arr = (Problem * len(self.probs))()
        for k, p in enumerate(self.probs):
            kx = torch.as_tensor(np.ascontiguousarray(p.kx), dtype=torch.float64, device=device)
            ky = torch.as_tensor(np.ascontiguousarray(p.ky), dtype=torch.float64, device=device)
            kz = torch.as_tensor(np.ascontiguousarray(p.kz), dtype=torch.float64, device=device)
            self._keep += [kx, ky, kz]
            arr[k] = Problem(p.dim, p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, kx.data_ptr(), ky.data_ptr(),
                             kz.data_ptr(), p.phi, p.mu_w, p.mu_n, p.rho_w, p.rho_n, p.g, p.pc_model,
                             p.pc_p0, p.pc_pd, p.bc_lambda, p.s_wr, p.s_nr, p.u_in, p.p_out, p.sn_out,
                             p.q_in, p.well_in, p.well_out)
        self.c = arr
        self.ncell = sum(p.ncell for p in self.probs)
        self.cell_off = np.cumsum([0] + [p.ncell for p in self.probs]).astype(np.int32)

    def __len__(self):
        return len(self.probs)


class Bsr2:
    """2x2-block CSR matrix in device memory (FP64)."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor,
                 seg_off: Optional[Sequence[int]] = None):
        self.row_ptr, self.col = row_ptr, col
        self.val = val
        self.nb = row_ptr.numel() - 1
        self.nnzb = col.numel()
        self.seg_off = None if seg_off is None else np.ascontiguousarray(seg_off, dtype=np.int32)

    @property
    def nseg(self):
        return 1 if self.seg_off is None else self.seg_off.size - 1

    def c(self):
        so = None if self.seg_off is None else self.seg_off.ctypes.data_as(C.c_void_p)
        return Bsr2C(self.nb, self.nnzb, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                     0 if self.seg_off is None else self.nseg, so)

    @classmethod
    def pattern(cls, dp: DeviceProblems, stream=None):
        nnzb = lib().rs_bsr2_nnzb(dp.c, len(dp))
        rp = torch.empty(dp.ncell + 1, dtype=torch.int32, device="cuda")
        col = torch.empty(nnzb, dtype=torch.int32, device="cuda")
        _check(lib().rs_bsr2_pattern(dp.c, len(dp), _ptr(rp), _ptr(col), _stream(stream)), "rs_bsr2_pattern")
        val = torch.zeros(4 * nnzb, dtype=torch.float64, device="cuda")
        return cls(rp, col, val, None if len(dp) == 1 else dp.cell_off)

    @classmethod
    def from_host(cls, row_ptr, col, val, seg_off=None):
        return cls(torch.as_tensor(np.ascontiguousarray(row_ptr, dtype=np.int32), device="cuda"),
                   torch.as_tensor(np.ascontiguousarray(col, dtype=np.int32), device="cuda"),
                   torch.as_tensor(np.ascontiguousarray(val, dtype=np.float64).reshape(-1), device="cuda"),
                   seg_off)


class Csr:
    def __init__(self, row_ptr, col, val, seg_off=None):
        self.row_ptr = torch.as_tensor(row_ptr, dtype=torch.int32, device="cuda").contiguous()
        self.col = torch.as_tensor(col, dtype=torch.int32, device="cuda").contiguous()
        self.val = torch.as_tensor(val, dtype=torch.float64, device="cuda").contiguous()
        self.n = self.row_ptr.numel() - 1
        self.seg_off = None if seg_off is None else np.ascontiguousarray(seg_off, dtype=np.int32)

    def c(self):
        so = None if self.seg_off is None else self.seg_off.ctypes.data_as(C.c_void_p)
        return CsrC(self.n, self.col.numel(), _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                    0 if self.seg_off is None else self.seg_off.size - 1, so)


# ------------------------------------------------------------------ params
@dataclass
class AmgParams:
    theta: float = 0.25
    seed: int = 20161101
    max_levels: int = 25
    coarse_n: int = 64
    max_dense: int = 2048
    smoother: int = 2
    nu1: int = 1
    nu2: int = 1
    interp: int = 1
    num_functions: int = 1
    precision: int = FP32
    chunk: int = 512
    agg_levels: int = 0
    chunk_coarse: int = 32
    restriction: int = 0

    def c(self):
        return AmgParamsC(self.theta, self.seed, self.max_levels, self.coarse_n, self.max_dense,
                          self.smoother, self.nu1, self.nu2, self.interp, self.num_functions,
                          self.precision, self.chunk, self.agg_levels, self.chunk_coarse,
                          self.restriction)


@dataclass
class PrecParams:
    kind: int = CPR1
    decouple: int = DECOUPLE_QIMPES
    p1: int = 0
    amg: AmgParams = field(default_factory=AmgParams)

    def c(self):
        return PrecParamsC(self.kind, self.decouple, self.p1, self.amg.c())


@dataclass
class GmresParams:
    m: int = 30
    maxit: int = 1000
    rtol: float = 1e-8

    def c(self):
        return GmresParamsC(self.m, self.maxit, self.rtol)


@dataclass
class GmresStats:
    status: int
    iterations: int
    converged: int
    relres: float
    its: np.ndarray
    relres_seg: np.ndarray


@dataclass
class NewtonParams:
    max_newton: int = 20
    ftol: float = 1e-6
    gmres: GmresParams = field(default_factory=GmresParams)
    prec: PrecParams = field(default_factory=PrecParams)
    max_ds: float = 0.0      # > 0: Appleyard chop of each cell's S_n change per iteration

    def c(self):
        return NewtonParamsC(self.max_newton, self.ftol, self.gmres.c(), self.prec.c(), self.max_ds)


# ------------------------------------------------------------------ calls
def jacobian_assemble(dp: DeviceProblems, u: torch.Tensor, u_old: torch.Tensor, dt: float,
                      J: Optional[Bsr2], F: torch.Tensor, stream=None):
    Jc = J.c() if J is not None else None
    _check(lib().jacobian_assemble(dp.c, len(dp), _ptr(u), _ptr(u_old), float(dt),
                                   C.byref(Jc) if Jc is not None else None, _ptr(F), _stream(stream)),
           "jacobian_assemble")


def jacobian_assemble_noalloc(dp: DeviceProblems, u: torch.Tensor, u_old: torch.Tensor, dt: float,
                              J: Optional[Bsr2], F: torch.Tensor, stream=None):
    """jacobian_assemble without device allocation (fixed scratch in the library)."""
    Jc = J.c() if J is not None else None
    _check(lib().jacobian_assemble_noalloc(dp.c, len(dp), _ptr(u), _ptr(u_old), float(dt),
                                           C.byref(Jc) if Jc is not None else None, _ptr(F), _stream(stream)),
           "jacobian_assemble_noalloc")


def bsr2_spmv(J: Bsr2, x: torch.Tensor, y: torch.Tensor, stream=None):
    _check(lib().bsr2_spmv(C.byref(J.c()), _ptr(x), _ptr(y), _stream(stream)), "bsr2_spmv")


def bsr2_residual(J: Bsr2, x, b, r, stream=None):
    _check(lib().bsr2_residual(C.byref(J.c()), _ptr(x), _ptr(b), _ptr(r), _stream(stream)), "bsr2_residual")


class Amg:
    """AMG hierarchy handle (owned unless it is a view into a preconditioner)."""

    def __init__(self, handle, owner=None, own=True):
        self.h = handle
        self._owner = owner
        self._own = own

    @classmethod
    def setup(cls, A: Csr, params: AmgParams = None, stream=None):
        params = params or AmgParams()
        h = C.c_void_p()
        Ac = A.c()
        _check(lib().amg_setup(C.byref(Ac), C.byref(params.c()), C.byref(h), _stream(stream)), "amg_setup")
        obj = cls(h, own=True)
        obj._A = A
        return obj

    def close(self):
        if self._own and self.h:
            lib().amg_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, b: torch.Tensor, x: torch.Tensor, stream=None):
        _check(lib().amg_apply(self.h, _ptr(b), _ptr(x), _stream(stream)), "amg_apply")

    @property
    def nlevels(self) -> int:
        n = C.c_int32()
        _check(lib().amg_levels(self.h, C.byref(n)), "amg_levels")
        return n.value

    def level_info(self, l: int):
        n, nnz, nnzp, nc = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().amg_level_info(self.h, l, C.byref(n), C.byref(nnz), C.byref(nnzp), C.byref(nc)),
               "amg_level_info")
        return n.value, nnz.value, nnzp.value, nc.value

    def level_smooth(self, l: int, sweeps: int, stream=None) -> float:
        """Run smoother sweeps on level l's own vectors; returns bytes per sweep."""
        by = C.c_double()
        _check(lib().amg_level_smooth(self.h, l, sweeps, C.byref(by), _stream(stream)), "amg_level_smooth")
        return by.value

    def level_transfer(self, l: int, which: int, reps: int, stream=None) -> float:
        """Launch a transfer kernel of level l `reps` times (0 residual, 1
        restriction, 2 prolongation); returns bytes per launch."""
        by = C.c_double()
        _check(lib().amg_level_transfer(self.h, l, which, reps, C.byref(by), _stream(stream)), "amg_level_transfer")
        return by.value

    def sizes(self) -> List[int]:
        return [self.level_info(l)[0] for l in range(self.nlevels)]

    def level(self, l: int, stream=None):
        """Level l as host numpy arrays: A (rp, col, val), cf, P (rp, col, val), colour."""
        n, nnz, nnzp, nc = self.level_info(l)
        d = "cuda"
        arp = torch.empty(n + 1, dtype=torch.int32, device=d)
        acol = torch.empty(max(nnz, 1), dtype=torch.int32, device=d)
        aval = torch.empty(max(nnz, 1), dtype=torch.float64, device=d)
        cf = torch.empty(max(n, 1), dtype=torch.int8, device=d)
        prp = torch.zeros(n + 1, dtype=torch.int32, device=d)
        pcol = torch.empty(max(nnzp, 1), dtype=torch.int32, device=d)
        pval = torch.empty(max(nnzp, 1), dtype=torch.float64, device=d)
        colour = torch.empty(max(n, 1), dtype=torch.int32, device=d)
        _check(lib().amg_level_copy(self.h, l, _ptr(arp), _ptr(acol), _ptr(aval), _ptr(cf), _ptr(prp),
                                    _ptr(pcol), _ptr(pval), _ptr(colour), _stream(stream)), "amg_level_copy")
        torch.cuda.current_stream().synchronize()
        out = dict(A=(arp.cpu().numpy(), acol.cpu().numpy()[:nnz], aval.cpu().numpy()[:nnz]),
                   cf=cf.cpu().numpy()[:n], colour=colour.cpu().numpy()[:n], ncolours=nc)
        if nnzp > 0 or l + 1 < self.nlevels:
            out["P"] = (prp.cpu().numpy(), pcol.cpu().numpy()[:nnzp], pval.cpu().numpy()[:nnzp])
        return out


class Precond:
    def __init__(self, J: Bsr2, params: PrecParams = None, stream=None):
        self.params = params or PrecParams()
        self.J = J
        self._Jc = J.c()
        self.h = C.c_void_p()
        _check(lib().precond_create(C.byref(self._Jc), C.byref(self.params.c()), C.byref(self.h),
                                    _stream(stream)), "precond_create")

    def close(self):
        if self.h:
            lib().precond_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, r: torch.Tensor, z: torch.Tensor, stream=None):
        _check(lib().precond_apply(self.h, _ptr(r), _ptr(z), _stream(stream)), "precond_apply")

    def amg(self, which: int) -> Optional[Amg]:
        h = lib().precond_amg(self.h, which)
        return Amg(C.c_void_p(h), owner=self, own=False) if h else None


class Ilu0:
    """ILU(0) of the point-ordered scalar matrix of J (P1 of CPR)."""

    def __init__(self, J: Bsr2, precision: int = FP64, stream=None):
        self.J = J
        self._Jc = J.c()
        self.h = C.c_void_p()
        _check(lib().ilu0_create(C.byref(self._Jc), precision, C.byref(self.h), _stream(stream)), "ilu0_create")

    def apply(self, b: torch.Tensor, x: torch.Tensor, stream=None):
        _check(lib().ilu0_apply(self.h, _ptr(b), _ptr(x), _stream(stream)), "ilu0_apply")

    def info(self):
        """(levels, widest level, CTAs per cluster)"""
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().ilu0_info(self.h, C.byref(a), C.byref(b), C.byref(c)), "ilu0_info")
        return a.value, b.value, c.value

    def factors(self, stream=None) -> torch.Tensor:
        lu = torch.empty_like(self.J.val)
        _check(lib().ilu0_factors(self.h, _ptr(lu), _stream(stream)), "ilu0_factors")
        return lu

    def close(self):
        if self.h:
            lib().ilu0_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gmres_solve(J: Bsr2, M: Optional[Precond], b: torch.Tensor, x: torch.Tensor,
                params: GmresParams = None, stream=None) -> GmresStats:
    params = params or GmresParams()
    its = np.zeros(J.nseg, dtype=np.int32)
    rr = np.zeros(J.nseg, dtype=np.float64)
    st = GmresStatsC(0, 0, 0.0, its.ctypes.data_as(C.c_void_p), rr.ctypes.data_as(C.c_void_p))
    Jc = J.c()
    rc = _check(lib().gmres_solve(C.byref(Jc), M.h if M is not None else None, _ptr(b), _ptr(x),
                                  C.byref(params.c()), C.byref(st), _stream(stream)), "gmres_solve")
    return GmresStats(rc, st.iterations, st.converged, st.relres, its, rr)


def newton_step(dp: DeviceProblems, u: torch.Tensor, u_old: torch.Tensor, dt: float,
                params: NewtonParams = None, stream=None):
    params = params or NewtonParams()
    st = NewtonStatsC()
    rc = _check(lib().newton_step(dp.c, len(dp), _ptr(u), _ptr(u_old), float(dt), C.byref(params.c()),
                                  C.byref(st), _stream(stream)), "newton_step")
    return rc, dict(newton_its=st.newton_its, linear_its=st.linear_its, fnorm=st.fnorm,
                    setup_ms=st.setup_ms, solve_ms=st.solve_ms, assemble_ms=st.assemble_ms)


PROFILE_CLASSES = ("hybrid_gs_sweep", "csr_resid_restrict_prolong", "bsr2_spmv", "gmres_cgs2",
                   "setup_spgemm", "setup_interp", "other")


def profile_begin():
    _check(lib().rs_profile_begin(), "rs_profile_begin")


def profile_end():
    """Per kernel class: (ms, algorithmic bytes, launches), timed with CUDA events."""
    k = len(PROFILE_CLASSES)
    ms = np.zeros(k)
    by = np.zeros(k)
    n = np.zeros(k, dtype=np.int64)
    lib().rs_profile_end(ms.ctypes.data_as(C.c_void_p), by.ctypes.data_as(C.c_void_p),
                         n.ctypes.data_as(C.c_void_p), k)
    return {PROFILE_CLASSES[i]: (float(ms[i]), float(by[i]), int(n[i])) for i in range(k)}


def wait_status(stream=None) -> int:
    """RS_OK, or RS_ETIMEOUT (the flag is then cleared) when a smoother CTA
    gave up waiting for its staging copies since the last check."""
    rc = lib().rs_wait_status(_stream(stream))
    if rc < 0 and rc != RS_ETIMEOUT:
        _check(rc, "rs_wait_status")
    return rc


def raise_wait_flag(stream=None):
    """Set the capped-wait flag without running a kernel (error-path tests)."""
    _check(lib().rs_raise_wait_flag(_stream(stream)), "rs_raise_wait_flag")


def launch_count() -> int:
    return int(lib().rs_launch_count())


def autotune_bsr2(J: Bsr2, x: torch.Tensor, y: torch.Tensor, stream=None) -> int:
    """Pick the fastest lanes-per-row for y = J x on this matrix; returns it."""
    best = C.c_int()
    Jc = J.c()
    _check(lib().rs_autotune_bsr2(C.byref(Jc), _ptr(x), _ptr(y), C.byref(best), _stream(stream)), "rs_autotune_bsr2")
    return best.value


def set_bsr2_lanes(lpr: int):
    _check(lib().rs_tune_set_bsr2_lpr(int(lpr)), "rs_tune_set_bsr2_lpr")

"""Plain FP64 CPU oracle of the paper's solver (arXiv:1611.00127).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the library under
``paper_1611_00127_gb300`` never imports it and shares no code with it.

The arithmetic lives in the C files next to this one (single-threaded, FP64,
no fused multiply-add); this module only compiles them with gcc and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRCS = ["oracle_physics.c", "oracle_sparse.c", "oracle_amg.c", "oracle_solve.c"]

AMG_J, CPR1, CPR2, BF, AMG_J_SCALAR = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``_build/liboracle.so`` (plain gcc, -O2)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB):
        lt = os.path.getmtime(_LIB)
        if all(os.path.getmtime(s) <= lt for s in srcs):
            return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp] + [os.path.join(_HERE, s) for s in _SRCS] + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("kx", C.c_void_p), ("ky", C.c_void_p), ("kz", C.c_void_p),
                ("phi", C.c_double), ("mu_w", C.c_double), ("mu_n", C.c_double),
                ("rho_w", C.c_double), ("rho_n", C.c_double), ("g", C.c_double),
                ("pc_model", C.c_int32), ("pc_p0", C.c_double), ("pc_pd", C.c_double),
                ("bc_lambda", C.c_double), ("s_wr", C.c_double), ("s_nr", C.c_double),
                ("u_in", C.c_double), ("p_out", C.c_double), ("sn_out", C.c_double),
                ("q_in", C.c_double), ("well_in", C.c_int32), ("well_out", C.c_int32)]


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nnz", C.c_int32),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class _AmgParams(C.Structure):
    _fields_ = [("theta", C.c_double), ("seed", C.c_uint64), ("max_levels", C.c_int32),
                ("coarse_n", C.c_int32), ("max_dense", C.c_int32), ("smoother", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("interp", C.c_int32),
                ("num_functions", C.c_int32), ("chunk", C.c_int32), ("agg_levels", C.c_int32),
                ("chunk_coarse", C.c_int32), ("restriction", C.c_int32)]


class _PrecParams(C.Structure):
    _fields_ = [("kind", C.c_int32), ("decouple", C.c_int32), ("p1", C.c_int32),
                ("amg", _AmgParams)]


class _NewtonParams(C.Structure):
    _fields_ = [("max_newton", C.c_int32), ("ftol", C.c_double), ("gmres_m", C.c_int32),
                ("gmres_maxit", C.c_int32), ("gmres_rtol", C.c_double), ("prec", _PrecParams),
                ("max_ds", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.c_void_p
        i32, f64, u64 = C.c_int32, C.c_double, C.c_uint64
        sig = {
            "or_bsr2_nnzb": (i32, [P]),
            "or_bsr2_pattern": (None, [P, P, P]),
            "or_assemble": (None, [P, P, P, f64, P, P, P, P]),
            "or_constitutive": (None, [P, f64, P]),
            "or_bsr2_spmv": (None, [i32, P, P, P, P, P]),
            "or_csr_new": (P, [i32, i32, i32, P, P, P]),
            "or_csr_free": (None, [P]),
            "or_csr_info": (None, [P, P]),
            "or_csr_copy": (None, [P, P, P, P]),
            "or_scalar_from_bsr2": (P, [i32, P, P, P]),
            "or_bsr2_part": (P, [i32, P, P, P, i32, i32]),
            "or_decouple_abf": (None, [i32, P, P, P, P]),
            "or_ilu0_bsr2": (None, [i32, P, P, P, P]),
            "or_ilu0_solve_bsr2": (None, [i32, P, P, P, P, P]),
            "or_simple_schur": (P, [P, P, P, P]),
            "or_transpose": (P, [P]),
            "or_spgemm": (P, [P, P]),
            "or_csr_spmv": (None, [P, P, P]),
            "or_splitmix64": (u64, [u64, u64]),
            "or_strength": (None, [P, f64, P]),
            "or_pmis": (None, [P, P, u64, i32, P]),
            "or_interp": (P, [P, P, P]),
            "or_interp_ext": (P, [P, P, P]),
            "or_galerkin": (P, [P, P]),
            "or_air_restriction": (P, [P, P, i32, P]),
            "or_jp_colour": (i32, [P, u64, i32, P]),
            "or_chunk_rows": (i32, [P, i32]),
            "or_chunk_colour": (i32, [P, i32, P]),
            "or_chunk_colour_pt": (i32, [P, i32, i32, P]),
            "or_func_part": (P, [P, i32, i32]),
            "or_amg_setup": (P, [P, P]),
            "or_amg_free": (None, [P]),
            "or_amg_nlevels": (i32, [P]),
            "or_amg_A": (P, [P, i32]),
            "or_amg_P": (P, [P, i32]),
            "or_amg_cf": (None, [P, i32, P]),
            "or_amg_colours": (i32, [P, i32, P]),
            "or_amg_vcycle": (None, [P, P, P]),
            "or_amg_smooth": (None, [P, i32, P, P]),
            "or_dense_lu": (i32, [i32, P, P]),
            "or_dense_lu_solve": (None, [i32, P, P, P, P]),
            "or_precond_create": (P, [i32, P, P, P, P]),
            "or_precond_free": (None, [P]),
            "or_precond_apply": (None, [P, P, P]),
            "or_precond_amg": (P, [P, i32]),
            "or_fgmres": (i32, [i32, P, P, P, P, P, P, i32, f64, i32, P, P]),
            "or_newton": (i32, [P, P, P, f64, P, P, P, P]),
            "or_scaled_fnorm": (f64, [P, P, f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class _Keep:
    """Holds numpy arrays alive while C code keeps raw pointers to them."""


def _problem(prob) -> tuple:
    keep = _Keep()
    keep.kx, keep.ky, keep.kz = _f64(prob.kx), _f64(prob.ky), _f64(prob.kz)
    s = _Problem(prob.dim, prob.nx, prob.ny, prob.nz, prob.hx, prob.hy, prob.hz,
                 keep.kx.ctypes.data, keep.ky.ctypes.data, keep.kz.ctypes.data,
                 prob.phi, prob.mu_w, prob.mu_n, prob.rho_w, prob.rho_n, prob.g,
                 prob.pc_model, prob.pc_p0, prob.pc_pd, prob.bc_lambda, prob.s_wr,
                 prob.s_nr, prob.u_in, prob.p_out, prob.sn_out, prob.q_in, prob.well_in, prob.well_out)
    return s, keep


# ------------------------------------------------------------------ matrices
class Csr:
    """Owning handle of an oracle CSR matrix."""

    def __init__(self, handle):
        self.h = handle

    @classmethod
    def from_arrays(cls, rowptr, col, val, m: Optional[int] = None):
        rowptr, col, val = _i32(rowptr), _i32(col), _f64(val)
        n = rowptr.size - 1
        m = n if m is None else m
        return cls(lib().or_csr_new(n, m, int(rowptr[-1]), _p(rowptr), _p(col), _p(val)))

    @classmethod
    def from_scipy(cls, A):
        A = A.tocsr()
        A.sort_indices()
        return cls.from_arrays(A.indptr, A.indices, A.data, A.shape[1])

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_csr_free(self.h)
            self.h = None

    def info(self):
        o = np.zeros(3, dtype=np.int32)
        lib().or_csr_info(self.h, _p(o))
        return int(o[0]), int(o[1]), int(o[2])

    def arrays(self):
        n, m, nnz = self.info()
        rp = np.zeros(n + 1, dtype=np.int32)
        c = np.zeros(max(nnz, 1), dtype=np.int32)
        v = np.zeros(max(nnz, 1), dtype=np.float64)
        lib().or_csr_copy(self.h, _p(rp), _p(c), _p(v))
        return rp, c[:nnz], v[:nnz]

    def scipy(self):
        import scipy.sparse as sp
        n, m, nnz = self.info()
        rp, c, v = self.arrays()
        return sp.csr_matrix((v, c, rp), shape=(n, m))


class _View(Csr):
    """Non-owning view (matrix owned by a hierarchy)."""

    def __init__(self, handle, owner):
        self.h = handle
        self._owner = owner

    def __del__(self):
        pass


# ------------------------------------------------------------------ physics
def bsr2_pattern(prob):
    s, keep = _problem(prob)
    nnzb = lib().or_bsr2_nnzb(C.byref(s))
    rowptr = np.zeros(prob.ncell + 1, dtype=np.int32)
    col = np.zeros(nnzb, dtype=np.int32)
    lib().or_bsr2_pattern(C.byref(s), _p(rowptr), _p(col))
    return rowptr, col


def assemble(prob, u, u_old, dt, pattern=None, jacobian=True):
    """Residual F [2N] and Jacobian blocks [nnzb, 2, 2] at u."""
    s, keep = _problem(prob)
    rowptr, col = pattern if pattern is not None else bsr2_pattern(prob)
    u, u_old = _f64(u), _f64(u_old)
    F = np.zeros(2 * prob.ncell)
    J = np.zeros((col.size, 2, 2)) if jacobian else None
    lib().or_assemble(C.byref(s), _p(u), _p(u_old), float(dt), _p(rowptr), _p(col),
                      _p(J) if jacobian else None, _p(F))
    return F, J, (rowptr, col)


def constitutive(prob, sn: float):
    """(lambda_w, lambda_n, dlambda_w/dS_n, dlambda_n/dS_n, P_c, dP_c/dS_n)."""
    s, keep = _problem(prob)
    o = np.zeros(6)
    lib().or_constitutive(C.byref(s), float(sn), _p(o))
    return o


def scaled_fnorm(prob, F, dt):
    s, keep = _problem(prob)
    return lib().or_scaled_fnorm(C.byref(s), _p(_f64(F)), float(dt))


def bsr2_spmv(rowptr, col, val, x):
    x = _f64(x)
    y = np.zeros_like(x)
    lib().or_bsr2_spmv(rowptr.size - 1, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), _p(x), _p(y))
    return y


def bsr2_to_scipy(rowptr, col, val):
    """Point-ordered scalar matrix (2N x 2N) of a 2x2 block matrix."""
    import scipy.sparse as sp
    nb = rowptr.size - 1
    return sp.bsr_matrix((np.asarray(val).reshape(-1, 2, 2), col, rowptr), shape=(2 * nb, 2 * nb)).tocsr()


def scalar_from_bsr2(rowptr, col, val) -> Csr:
    return Csr(lib().or_scalar_from_bsr2(rowptr.size - 1, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val))))


def bsr2_part(rowptr, col, val, r, c) -> Csr:
    return Csr(lib().or_bsr2_part(rowptr.size - 1, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), r, c))


def decouple_abf(rowptr, col, val):
    val = _f64(val)
    out = np.zeros_like(val)
    lib().or_decouple_abf(rowptr.size - 1, _p(_i32(rowptr)), _p(_i32(col)), _p(val), _p(out))
    return out


def ilu0(rowptr, col, val):
    """ILU(0) factors of the point-ordered scalar matrix, in the block layout."""
    val = _f64(val)
    lu = np.zeros_like(val)
    lib().or_ilu0_bsr2(rowptr.size - 1, _p(_i32(rowptr)), _p(_i32(col)), _p(val), _p(lu))
    return lu


def ilu0_solve(rowptr, col, lu, b):
    b = _f64(b)
    x = np.zeros_like(b)
    lib().or_ilu0_solve_bsr2(rowptr.size - 1, _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(lu)), _p(b), _p(x))
    return x


def simple_schur(App: Csr, Aps: Csr, Asp: Csr, Ass: Csr) -> Csr:
    return Csr(lib().or_simple_schur(App.h, Aps.h, Asp.h, Ass.h))


def spgemm(A: Csr, B: Csr) -> Csr:
    return Csr(lib().or_spgemm(A.h, B.h))


def transpose(A: Csr) -> Csr:
    return Csr(lib().or_transpose(A.h))


# ------------------------------------------------------------------ AMG
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
    chunk: int = 512
    agg_levels: int = 0
    chunk_coarse: int = 32
    restriction: int = 0

    def c(self):
        return _AmgParams(self.theta, self.seed, self.max_levels, self.coarse_n,
                          self.max_dense, self.smoother, self.nu1, self.nu2, self.interp,
                          self.num_functions, self.chunk, self.agg_levels, self.chunk_coarse, self.restriction)


def splitmix64(seed: int, counter: int) -> int:
    return int(lib().or_splitmix64(seed, counter))


def strength(A: Csr, theta: float):
    n, m, nnz = A.info()
    s = np.zeros(max(nnz, 1), dtype=np.uint8)
    lib().or_strength(A.h, float(theta), _p(s))
    return s[:nnz]


def pmis(A: Csr, strong, seed: int, level: int = 0):
    n, m, nnz = A.info()
    cf = np.zeros(n, dtype=np.int8)
    lib().or_pmis(A.h, _p(np.ascontiguousarray(strong, dtype=np.uint8)), seed, level, _p(cf))
    return cf


def interp(A: Csr, strong, cf) -> Csr:
    return Csr(lib().or_interp(A.h, _p(np.ascontiguousarray(strong, dtype=np.uint8)),
                               _p(np.ascontiguousarray(cf, dtype=np.int8))))


def interp_ext(A: Csr, strong, cf) -> Csr:
    return Csr(lib().or_interp_ext(A.h, _p(np.ascontiguousarray(strong, dtype=np.uint8)),
                                   _p(np.ascontiguousarray(cf, dtype=np.int8))))


def air_restriction(A: Csr, cf, dist: int = 1, strong=None) -> Csr:
    """Approximate ideal restriction for the splitting cf (rows: C points);
    with `strong` (one flag per entry of A) over strong couplings only."""
    st = None if strong is None else np.ascontiguousarray(strong, dtype=np.uint8)
    return Csr(lib().or_air_restriction(A.h, _p(np.ascontiguousarray(cf, dtype=np.int8)), int(dist),
                                        None if st is None else _p(st)))


def galerkin(A: Csr, P: Csr) -> Csr:
    return Csr(lib().or_galerkin(A.h, P.h))


def jp_colour(A: Csr, seed: int, level: int = 0):
    n, m, nnz = A.info()
    col = np.zeros(n, dtype=np.int32)
    nc = lib().or_jp_colour(A.h, seed, level, _p(col))
    return col, int(nc)


def chunk_colour(A: Csr, chunk: int = 512):
    n, m, nnz = A.info()
    col = np.zeros(n, dtype=np.int32)
    nc = lib().or_chunk_colour(A.h, chunk, _p(col))
    return col, int(nc), int(lib().or_chunk_rows(A.h, chunk))


def chunk_colour_pt(A: Csr, chunk: int = 512, b: int = 2):
    """Point colouring of the point-block hybrid smoother (colour per row)."""
    n, m, nnz = A.info()
    col = np.zeros(n, dtype=np.int32)
    nc = lib().or_chunk_colour_pt(A.h, chunk, b, _p(col))
    return col, int(nc)


def func_part(A: Csr, b: int, f: int) -> Csr:
    """Rows b*i + f and columns b*j + f of A."""
    return Csr(lib().or_func_part(A.h, b, f))


class Amg:
    def __init__(self, A: Csr, params: AmgParams = None, _handle=None, _owner=None):
        self.params = params or AmgParams()
        if _handle is not None:
            self.h, self._owner, self._own = _handle, _owner, False
        else:
            self._A = A
            self.h, self._own = lib().or_amg_setup(A.h, C.byref(self.params.c())), True

    def __del__(self):
        if getattr(self, "_own", False) and _lib is not None and self.h:
            _lib.or_amg_free(self.h)
            self.h = None

    @property
    def nlevels(self) -> int:
        return int(lib().or_amg_nlevels(self.h))

    def A(self, l) -> Csr:
        return _View(lib().or_amg_A(self.h, l), self)

    def P(self, l) -> Csr:
        return _View(lib().or_amg_P(self.h, l), self)

    def cf(self, l):
        n = self.A(l).info()[0]
        out = np.zeros(n, dtype=np.int8)
        lib().or_amg_cf(self.h, l, _p(out))
        return out

    def colours(self, l):
        n = self.A(l).info()[0]
        out = np.zeros(n, dtype=np.int32)
        nc = lib().or_amg_colours(self.h, l, _p(out))
        return out, int(nc)

    def sizes(self):
        return [self.A(l).info()[0] for l in range(self.nlevels)]

    def vcycle(self, b):
        b = _f64(b)
        x = np.zeros_like(b)
        lib().or_amg_vcycle(self.h, _p(b), _p(x))
        return x

    def smooth(self, l, b, x):
        b, x = _f64(b), _f64(x).copy()
        lib().or_amg_smooth(self.h, l, _p(b), _p(x))
        return x


def dense_lu_solve(A, b):
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    n = a.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    lib().or_dense_lu(n, _p(a), _p(piv))
    x = np.zeros(n)
    lib().or_dense_lu_solve(n, _p(a), _p(piv), _p(_f64(b)), _p(x))
    return x


# ------------------------------------------------------------------ solvers
@dataclass
class PrecParams:
    kind: int = CPR1
    decouple: int = 1
    p1: int = 0
    amg: AmgParams = None

    def c(self):
        return _PrecParams(self.kind, self.decouple, self.p1, (self.amg or AmgParams()).c())


class Precond:
    def __init__(self, rowptr, col, val, params: PrecParams):
        self.rowptr, self.col, self.val = _i32(rowptr), _i32(col), _f64(val)
        self.params = params
        self.nb = self.rowptr.size - 1
        self.h = lib().or_precond_create(self.nb, _p(self.rowptr), _p(self.col), _p(self.val),
                                         C.byref(params.c()))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_precond_free(self.h)
            self.h = None

    def apply(self, r):
        r = _f64(r)
        z = np.zeros_like(r)
        lib().or_precond_apply(self.h, _p(r), _p(z))
        return z

    def amg(self, which: int) -> Optional[Amg]:
        h = lib().or_precond_amg(self.h, which)
        return Amg(None, self.params.amg, _handle=h, _owner=self) if h else None


def fgmres(rowptr, col, val, b, M: Optional[Precond] = None, x0=None, m=30, rtol=1e-8, maxit=1000):
    """Returns (x, status, iterations, relres)."""
    rowptr, col, val, b = _i32(rowptr), _i32(col), _f64(val), _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    its = C.c_int32(0)
    rr = C.c_double(0.0)
    st = lib().or_fgmres(rowptr.size - 1, _p(rowptr), _p(col), _p(val), M.h if M else None,
                         _p(b), _p(x), m, rtol, maxit, C.byref(its), C.byref(rr))
    return x, int(st), int(its.value), float(rr.value)


@dataclass
class NewtonParams:
    max_newton: int = 20
    ftol: float = 1e-6
    gmres_m: int = 30
    gmres_maxit: int = 1000
    gmres_rtol: float = 1e-8
    prec: PrecParams = None
    max_ds: float = 0.0

    def c(self):
        return _NewtonParams(self.max_newton, self.ftol, self.gmres_m, self.gmres_maxit,
                             self.gmres_rtol, (self.prec or PrecParams()).c(), self.max_ds)


def newton(prob, u, u_old, dt, params: NewtonParams = None):
    """One backward-Euler step; returns (u_new, status, newton_its, linear_its, fnorm_hist)."""
    params = params or NewtonParams()
    s, keep = _problem(prob)
    u = _f64(u).copy()
    u_old = _f64(u_old)
    ni, li = C.c_int32(0), C.c_int32(0)
    hist = np.full(params.max_newton + 1, np.nan)
    st = lib().or_newton(C.byref(s), _p(u), _p(u_old), float(dt), C.byref(params.c()),
                         C.byref(ni), C.byref(li), _p(hist))
    return u, int(st), int(ni.value), int(li.value), hist[: ni.value + 1]

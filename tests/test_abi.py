"""The C-ABI library builds, loads and exports every function include/rsflow.h
declares (no GPU work)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rsflow.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "sizeof")))


def test_library_exports_every_declared_symbol():
    from paper_1611_00127_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 18, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_string_without_gpu():
    from paper_1611_00127_gb300 import rsflow as R
    L = R.lib()
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.rs_version(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == 0
    assert c.value == 103
    assert isinstance(L.rs_last_error(), bytes)


def test_nnzb_host_count_matches_oracle_pattern(oracle, inputs):
    """rs_bsr2_nnzb is pure host arithmetic: compare with the oracle pattern."""
    from paper_1611_00127_gb300 import rsflow as R
    for p in (inputs.config_small_2d(), inputs.homogeneous(5, 4, nz=3), inputs.homogeneous(1, 7)):
        arr = (R.Problem * 1)()
        arr[0] = R.Problem(p.dim, p.nx, p.ny, p.nz, p.hx, p.hy, p.hz, 0, 0, 0, p.phi, p.mu_w, p.mu_n, p.rho_w,
                           p.rho_n, p.g, p.pc_model, p.pc_p0, p.pc_pd, p.bc_lambda, p.s_wr, p.s_nr, p.u_in,
                           p.p_out, p.sn_out)
        rp, col = oracle.bsr2_pattern(p)
        assert R.lib().rs_bsr2_nnzb(arr, 1) == col.size


def test_invalid_arguments_rejected_on_host():
    """Argument validation happens before any GPU work."""
    from paper_1611_00127_gb300 import rsflow as R
    L = R.lib()
    h = ctypes.c_void_p()
    assert L.precond_create(None, None, ctypes.byref(h), None) == -1
    assert L.amg_setup(None, None, ctypes.byref(h), None) == -1
    assert L.gmres_solve(None, None, None, None, None, None, None) == -1
    assert b"invalid" in L.rs_last_error() or b"null" in L.rs_last_error()
    assert L.ilu0_create(None, 1, ctypes.byref(h), None) == -1
    assert L.ilu0_create(None, 1, None, None) == -1
    J = R.Bsr2C(0, 0, None, None, None, 0, None)
    assert L.ilu0_create(ctypes.byref(J), 5, ctypes.byref(h), None) == -1
    assert b"precision" in L.rs_last_error()
    assert L.ilu0_apply(None, None, None, None) == -1
    assert L.ilu0_info(None, None, None, None) == -1
    assert L.ilu0_factors(None, None, None) == -1
    assert L.ilu0_destroy(None) == 0
    n = ctypes.c_int32()
    assert L.amg_tail_level(None, ctypes.byref(n)) == -1


def test_parameter_validation_on_host():
    """Out-of-range solver parameters are refused with RS_EINVAL (-1) and a
    message naming the parameter, before any GPU work (an empty matrix is
    enough)."""
    from paper_1611_00127_gb300 import rsflow as R
    L = R.lib()
    csr = R.CsrC(0, 0, None, None, None, 0, None)
    bad = [(dict(agg_levels=9), b"agg_levels"), (dict(chunk_coarse=16), b"chunk_coarse"),
           (dict(tail_rows=-1), b"tail_rows"), (dict(theta=2.0), b"theta"),
           (dict(num_functions=3), b"num_functions"), (dict(precision=5), b"precision"),
           (dict(nu1=17), b"sweep"), (dict(chunk=16), b"chunk"), (dict(restriction=2), b"restriction")]
    for kw, word in bad:
        p = R.AmgParams(**kw).c()
        h = ctypes.c_void_p()
        assert L.amg_setup(ctypes.byref(csr), ctypes.byref(p), ctypes.byref(h), None) == -1, kw
        assert word in L.rs_last_error(), (kw, L.rs_last_error())
    J = R.Bsr2C(0, 0, None, None, None, 0, None)
    for kw, word in ((dict(kind=9), b"kind"), (dict(decouple=7), b"decoupling"), (dict(p1=2), b"P1")):
        pp = R.PrecParams(**kw).c()
        h = ctypes.c_void_p()
        assert L.precond_create(ctypes.byref(J), ctypes.byref(pp), ctypes.byref(h), None) == -1, kw
        assert word in L.rs_last_error(), (kw, L.rs_last_error())

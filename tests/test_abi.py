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


def test_parameter_validation_on_host():
    """Out-of-range solver parameters are refused with RS_EINVAL (-1) and a
    message naming the parameter, before any GPU work (an empty matrix is
    enough)."""
    from paper_1611_00127_gb300 import rsflow as R
    L = R.lib()
    csr = R.CsrC(0, 0, None, None, None, 0, None)
    bad = [(dict(agg_levels=9), b"agg_levels"), (dict(chunk_coarse=16), b"chunk_coarse"),
           (dict(theta=2.0), b"theta"),
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


def test_grid_sizes_checked_in_64_bit_before_any_launch():
    """A grid whose cell count wraps in 32-bit arithmetic (65537 x 65536
    wraps to 65536; 65536 x 65536 x 2 wraps to 0) is refused by every call
    that takes grid descriptions, before any GPU work, and so is a total
    beyond the 32-bit block index range. The vectors are host dummies that a
    refused call never touches."""
    from paper_1611_00127_gb300 import rsflow as R
    L = R.lib()
    buf = (ctypes.c_double * 4)()
    ibuf = (ctypes.c_int32 * 4)()
    cases = [(3, 65537, 65536, 1), (3, 65536, 65536, 2), (2, 1 << 30, 1, 1), (3, 1024, 1024, 1024)]
    for dim, nx, ny, nz in cases:
        arr = (R.Problem * 1)()
        arr[0] = R.Problem(dim, nx, ny, nz, 1.0, 1.0, 1.0, 0, 0, 0, 0.2, 1e-3, 5e-3, 1000.0, 700.0, 0.0,
                           2, 0.0, 5e3, 2.0, 0.0, 0.0, 1e-6, 1e5, 0.1, 0.0, -1, -1)
        ptr = ctypes.cast(buf, ctypes.c_void_p)
        assert L.jacobian_assemble(arr, 1, ptr, ptr, 86400.0, None, ptr, None) == -1, (nx, ny, nz)
        assert b"too many cells" in L.rs_last_error(), L.rs_last_error()
        assert L.jacobian_assemble_noalloc(arr, 1, ptr, ptr, 86400.0, None, ptr, None) == -1, (nx, ny, nz)
        assert b"too many cells" in L.rs_last_error(), L.rs_last_error()
        ip = ctypes.cast(ibuf, ctypes.c_void_p)
        assert L.rs_bsr2_pattern(arr, 1, ip, ip, None) == -1, (nx, ny, nz)
        assert b"too many cells" in L.rs_last_error(), L.rs_last_error()
    # two grids that fit alone but not together (dummy permeability pointers:
    # the first grid passes its own checks)
    buf_addr = ctypes.addressof(buf)
    arr = (R.Problem * 2)()
    for k in range(2):
        arr[k] = R.Problem(3, 1024, 1024, 600, 1.0, 1.0, 1.0, buf_addr, buf_addr, buf_addr, 0.2, 1e-3, 5e-3, 1000.0, 700.0, 0.0,
                           2, 0.0, 5e3, 2.0, 0.0, 0.0, 1e-6, 1e5, 0.1, 0.0, -1, -1)
    ptr = ctypes.cast(buf, ctypes.c_void_p)
    assert L.jacobian_assemble(arr, 2, ptr, ptr, 86400.0, None, ptr, None) == -1
    assert b"too many cells" in L.rs_last_error(), L.rs_last_error()

"""GPU (CUDA library through the C-ABI) against the CPU oracle.

Tolerances:
  * bit-exact: block pattern, C/F splittings, colourings, hierarchy patterns
    and FP64 setup values (same operation order on both sides, no FMA);
  * FP64 kernels with a different summation order (SpMV, assembly with the
    device pow, FP64 V-cycle): relative 1e-12 .. 1e-10 of the row/vector scale;
  * FGMRES solutions: true relative residual <= rtol = 1e-8 evaluated by the
    oracle in FP64, and relative error <= 1e-6 against the oracle's solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1611_00127_gb300 import rsflow
    rsflow.lib()
    return rsflow


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _small_cases(I):
    rng = np.random.default_rng(5)
    k = np.exp(rng.normal(np.log(1e-12), 1.0, 7 * 5 * 4))
    p3 = I.Problem(dim=3, nx=7, ny=5, nz=4, kx=k, ky=k * 0.5, kz=k * 0.1, pc_model=2, pc_pd=5e3, g=9.81)
    # point wells (corner injection cell, single-cell outlet) with gravity
    pw = I.config_small_2d().with_(pc_model=2, pc_pd=2e4, g=9.81, q_in=5.0 / 86400.0, well_in=0)
    pw = pw.with_(well_out=pw.nx - 1)
    p3w = p3.with_(q_in=1e-5, well_in=3 * 7 * 5 + 2 * 7, well_out=6)
    return [I.config_small_2d(), I.config_lognormal_2d(1e4, n=48), p3,
            I.config_small_2d().with_(pc_model=1, pc_p0=1e5, nx=13, ny=11, kx=np.full(143, 2e-12),
                                      ky=np.full(143, 1e-12), kz=np.full(143, 1e-12)), pw, p3w]


@pytest.mark.parametrize("case", range(6))
def test_assembly_matches_oracle(R, oracle, inputs, case):
    p = _small_cases(inputs)[case]
    u, uo = inputs.front_state(p)
    u = inputs.jitter(u, 3)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    dp = R.DeviceProblems(p)
    J = R.Bsr2.pattern(dp)
    F = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(u), _dev(uo), inputs.DAY, J, F)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(J.row_ptr.cpu().numpy(), rp)
    np.testing.assert_array_equal(J.col.cpu().numpy(), col)
    Jg = J.val.cpu().numpy().reshape(-1, 2, 2)
    np.testing.assert_allclose(Jg, Jo, rtol=1e-11, atol=1e-13 * np.abs(Jo).max())
    np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=1e-10, atol=1e-12 * np.abs(Fo).max())


def test_assembly_batch_of_grids(R, oracle, inputs):
    probs = _small_cases(inputs)
    us, uos = zip(*[inputs.front_state(p) for p in probs])
    dp = R.DeviceProblems(probs)
    J = R.Bsr2.pattern(dp)
    F = torch.empty(2 * dp.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(np.concatenate(us)), _dev(np.concatenate(uos)), inputs.DAY, J, F)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()
    off = dp.cell_off
    for k, p in enumerate(probs):
        Fo, Jo, _ = oracle.assemble(p, us[k], uos[k], inputs.DAY)
        np.testing.assert_allclose(Fg[2 * off[k]:2 * off[k + 1]], Fo, rtol=1e-10, atol=1e-12 * np.abs(Fo).max())


def test_bsr2_spmv_and_residual(R, oracle, inputs):
    for p in _small_cases(inputs):
        u, uo = inputs.front_state(p)
        Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
        J = R.Bsr2.from_host(rp, col, Jo)
        x = inputs.rhs_vector(2 * p.ncell, 1)
        b = inputs.rhs_vector(2 * p.ncell, 2)
        y = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
        for lanes in (1, 2, 4, 8):
            R.set_bsr2_lanes(lanes)
            R.bsr2_spmv(J, _dev(x), y)
            yo = oracle.bsr2_spmv(rp, col, Jo, x)
            np.testing.assert_allclose(y.cpu().numpy(), yo, rtol=1e-12, atol=1e-14 * np.abs(yo).max())
        R.set_bsr2_lanes(4)
        r = torch.empty_like(y)
        R.bsr2_residual(J, _dev(x), _dev(b), r)
        np.testing.assert_allclose(r.cpu().numpy(), b - yo, rtol=1e-12, atol=1e-14 * np.abs(yo).max())


def _hier_compare(gh, oh, exact_values=True):
    assert gh.nlevels == oh.nlevels, (gh.sizes(), oh.sizes())
    assert gh.sizes() == oh.sizes()
    for l in range(oh.nlevels):
        g = gh.level(l)
        orp, ocol, oval = oh.A(l).arrays()
        np.testing.assert_array_equal(g["A"][0], orp)
        np.testing.assert_array_equal(g["A"][1], ocol)
        if exact_values:
            np.testing.assert_array_equal(g["A"][2], oval)
        if l + 1 < oh.nlevels:
            np.testing.assert_array_equal(g["cf"], oh.cf(l))
            prp, pcol, pval = oh.P(l).arrays()
            np.testing.assert_array_equal(g["P"][0], prp)
            np.testing.assert_array_equal(g["P"][1], pcol)
            if exact_values:
                np.testing.assert_array_equal(g["P"][2], pval)
            col, nc = oh.colours(l)
            assert g["ncolours"] == nc
            np.testing.assert_array_equal(g["colour"], col)


def _amg_pair(R, oracle, rp, c, v, theta=0.25, interp=1, coarse_n=64, nfun=1, smoother=0):
    op = oracle.AmgParams(theta=theta, interp=interp, coarse_n=coarse_n, num_functions=nfun, smoother=smoother)
    gp = R.AmgParams(theta=theta, interp=interp, coarse_n=coarse_n, num_functions=nfun, smoother=smoother,
                     precision=R.FP64)
    oh = oracle.Amg(oracle.Csr.from_arrays(rp, c, v), op)
    gh = R.Amg.setup(R.Csr(rp, c, v), gp)
    return gh, oh


@pytest.mark.parametrize("interp", [0, 1])
def test_hierarchy_bit_exact_poisson(R, oracle, inputs, interp):
    for rp, c, v, th in ((*inputs.poisson_2d(40), 0.25), (*inputs.poisson_3d(14), 0.5)):
        gh, oh = _amg_pair(R, oracle, rp, c, v, theta=th, interp=interp)
        _hier_compare(gh, oh)


@pytest.mark.parametrize("which", ["App", "Ass", "Stilde", "J", "Jnf2"])
def test_hierarchy_bit_exact_jacobian_blocks(R, oracle, inputs, which):
    p = inputs.config_lognormal_2d(1e4, n=40)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    nf = 1
    if which == "App":
        A = oracle.bsr2_part(rp, col, oracle.decouple_abf(rp, col, Jo), 0, 0)
    elif which == "Ass":
        A = oracle.bsr2_part(rp, col, Jo, 1, 1)
    elif which == "Stilde":
        A = oracle.simple_schur(*[oracle.bsr2_part(rp, col, Jo, r, c) for r, c in ((0, 0), (0, 1), (1, 0), (1, 1))])
    else:
        A = oracle.scalar_from_bsr2(rp, col, Jo)
        nf = 2 if which == "Jnf2" else 1
    arp, ac, av = A.arrays()
    gh, oh = _amg_pair(R, oracle, arp, ac, av, nfun=nf)
    _hier_compare(gh, oh)


def test_precond_hierarchies_bit_exact(R, oracle, inputs):
    """Hierarchies built inside the preconditioners (decoupling, SIMPLE Schur
    on the device) match the oracle's from the same J."""
    p = inputs.config_lognormal_2d(1e3, n=36)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    for kind, dec in ((1, 2), (1, 1), (2, 2), (3, 0), (0, 0), (4, 0)):
        gM = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=R.FP64)))
        oM = oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec))
        _hier_compare(gM.amg(0), oM.amg(0))
        if kind in (2, 3):
            _hier_compare(gM.amg(1), oM.amg(1))


@pytest.mark.parametrize("smoother", [0, 1, 2])
def test_vcycle_fp64_matches_oracle(R, oracle, inputs, smoother):
    rp, c, v = inputs.poisson_2d(50)
    gh, oh = _amg_pair(R, oracle, rp, c, v, smoother=smoother)
    b = inputs.rhs_vector(2500, 9)
    x = torch.empty(2500, dtype=torch.float64, device="cuda")
    gh.apply(_dev(b), x)
    xo = oh.vcycle(b)
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=1e-10, atol=1e-11 * np.abs(xo).max())


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_point_vcycle_matches_oracle(R, oracle, inputs, prec):
    """Systems (point) AMG on the scalar two-phase J: point coarsening,
    interleaved interpolation and the point-block hybrid smoother give the
    oracle's V-cycle (FP64 to 1e-10, FP32 to 1e-5)."""
    p = inputs.config_lognormal_2d(1e4, n=40)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    arp, ac, av = oracle.scalar_from_bsr2(rp, col, Jo).arrays()
    oh = oracle.Amg(oracle.Csr.from_arrays(arp, ac, av), oracle.AmgParams(num_functions=2))
    gh = R.Amg.setup(R.Csr(arp, ac, av), R.AmgParams(num_functions=2, precision=getattr(R, prec)))
    _hier_compare(gh, oh)
    b = -Fo
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    gh.apply(_dev(b), x)
    xo = oh.vcycle(b)
    xg = x.cpu().numpy()
    for comp in (0, 1):
        a, e = xg[comp::2], xo[comp::2]
        if prec == "FP64":
            np.testing.assert_allclose(a, e, rtol=1e-10, atol=1e-11 * np.abs(e).max())
        else:
            assert np.linalg.norm(a - e) / np.linalg.norm(e) < 1e-5


def test_vcycle_fp32_close_to_oracle(R, oracle, inputs):
    rp, c, v = inputs.poisson_2d(50)
    oh = oracle.Amg(oracle.Csr.from_arrays(rp, c, v))
    gh = R.Amg.setup(R.Csr(rp, c, v), R.AmgParams(precision=R.FP32))
    b = inputs.rhs_vector(2500, 9)
    x = torch.empty(2500, dtype=torch.float64, device="cuda")
    gh.apply(_dev(b), x)
    xo = oh.vcycle(b)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-5


@pytest.mark.parametrize("kind,dec", [(0, 0), (1, 0), (1, 1), (1, 2), (2, 2), (3, 0)])
def test_precond_apply_fp64_matches_oracle(R, oracle, inputs, kind, dec):
    p = inputs.config_small_2d()
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    gM = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=R.FP64)))
    oM = oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec))
    r = -Fo
    z = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    gM.apply(_dev(r), z)
    zo = oM.apply(r)
    zg = z.cpu().numpy()
    for comp in (0, 1):
        a, b = zg[comp::2], zo[comp::2]
        np.testing.assert_allclose(a, b, rtol=1e-8, atol=1e-9 * np.abs(b).max())


def _solve_pair(R, oracle, inputs, p, kind, dec, prec, rtol=1e-8, maxit=600):
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    b = -Fo
    x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
    M = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=prec)))
    st = R.gmres_solve(J, M, _dev(b), x, R.GmresParams(rtol=rtol, maxit=maxit))
    xg = x.cpu().numpy()
    return st, xg, (rp, col, Jo, b)


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
@pytest.mark.parametrize("kind,dec", [(0, 0), (1, 2), (1, 1), (1, 0), (2, 2), (3, 0)])
def test_gmres_solution_matches_oracle(R, oracle, inputs, prec, kind, dec):
    p = inputs.config_small_2d()
    st, xg, (rp, col, Jo, b) = _solve_pair(R, oracle, inputs, p, kind, dec, getattr(R, prec))
    assert st.status == R.RS_OK, st
    res = b - oracle.bsr2_spmv(rp, col, Jo, xg)
    assert np.linalg.norm(res) <= 1.0e-8 * np.linalg.norm(b) * 1.0001
    xo, sto, _, _ = oracle.fgmres(rp, col, Jo, b, oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec)))
    assert sto == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6


def test_gmres_unpreconditioned_and_zero_rhs(R, oracle, inputs):
    p = inputs.homogeneous(6, 5).with_(pc_model=2, pc_pd=5e3)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
    st = R.gmres_solve(J, None, _dev(-Fo), x, R.GmresParams(m=60, rtol=1e-10, maxit=60))
    assert st.status == R.RS_OK
    A = oracle.bsr2_to_scipy(rp, col, Jo).toarray()
    np.testing.assert_allclose(x.cpu().numpy(), np.linalg.solve(A, -Fo), rtol=1e-6)
    # zero right-hand side: converged at once with x = 0
    x0 = torch.zeros_like(x)
    st = R.gmres_solve(J, None, torch.zeros_like(x), x0, R.GmresParams())
    assert st.status == R.RS_OK and st.iterations == 0 and float(x0.abs().max()) == 0.0


@pytest.mark.parametrize("kind", ["BF", "AMG_J"])
def test_batch_equals_single_systems(R, oracle, inputs, kind):
    """Three systems of different sizes solved in one batch: each solution
    meets the tolerance (by the oracle's residual) and matches the single
    solve to the parity bar. The smoother's lanes per row are tuned per level
    shape, and a stacked level may get another choice than a single system's,
    so the FP32 V-cycle's summation order can differ: iteration counts agree
    within one."""
    probs = [inputs.config_lognormal_2d(1e4, n=24, member=1), inputs.config_small_2d(),
             inputs.config_lognormal_2d(1e3, n=40, member=2)]
    dp = R.DeviceProblems(probs)
    J = R.Bsr2.pattern(dp)
    us, uos = zip(*[inputs.front_state(p) for p in probs])
    F = torch.empty(2 * dp.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(np.concatenate(us)), _dev(np.concatenate(uos)), inputs.DAY, J, F)
    b = -F
    x = torch.zeros_like(b)
    prm = R.PrecParams(kind=getattr(R, kind), decouple=0, amg=R.AmgParams(precision=R.FP32))
    M = R.Precond(J, prm)
    st = R.gmres_solve(J, M, b, x, R.GmresParams())
    assert st.status == R.RS_OK and st.converged == 3
    xb = x.cpu().numpy()
    off = dp.cell_off
    Hb = M.amg(0)
    for k, p in enumerate(probs):
        dpk = R.DeviceProblems(p)
        Jk = R.Bsr2.pattern(dpk)
        Fk = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
        R.jacobian_assemble(dpk, _dev(us[k]), _dev(uos[k]), inputs.DAY, Jk, Fk)
        Mk = R.Precond(Jk, prm)
        xk = torch.zeros_like(Fk)
        stk = R.gmres_solve(Jk, Mk, -Fk, xk, R.GmresParams())
        assert abs(int(st.its[k]) - stk.iterations) <= 1
        xs = xk.cpu().numpy()
        assert np.linalg.norm(xb[2 * off[k]:2 * off[k + 1]] - xs) <= 1e-6 * np.linalg.norm(xs)
        Fo, Jo, (rp, col) = oracle.assemble(p, us[k], uos[k], inputs.DAY)
        res = -Fo - oracle.bsr2_spmv(rp, col, Jo, xb[2 * off[k]:2 * off[k + 1]])
        assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(Fo) * 1.01
    assert Hb.nlevels >= 2


def test_newton_step_matches_oracle(R, oracle, inputs):
    p = inputs.config_small_2d()
    u0 = inputs.initial_state(p)
    prm = R.NewtonParams(prec=R.PrecParams(kind=R.CPR1, amg=R.AmgParams(precision=R.FP32)))
    dp = R.DeviceProblems(p)
    ud = _dev(u0)
    rc, st = R.newton_step(dp, ud, _dev(u0), inputs.DAY, prm)
    assert rc == R.RS_OK, st
    uo, sto, ni, li, hist = oracle.newton(p, u0, u0, inputs.DAY,
                                          oracle.NewtonParams(prec=oracle.PrecParams(kind=1, decouple=2)))
    assert sto == 0
    ug = ud.cpu().numpy()
    F, _, _ = oracle.assemble(p, ug, u0, inputs.DAY, jacobian=False)
    assert oracle.scaled_fnorm(p, F, inputs.DAY) <= 1e-6
    np.testing.assert_allclose(ug[0::2], uo[0::2], rtol=1e-7)
    np.testing.assert_allclose(ug[1::2], uo[1::2], atol=1e-7)


def test_precond_hierarchies_bit_exact_3d(R, oracle, inputs):
    """3D layered field (7-point J, dense coarse rows): the CPR and BF
    hierarchies built on the device match the oracle's bit for bit."""
    p = inputs.config_layered_3d(n=16, layers=4)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    for kind, dec in ((1, 2), (3, 0), (0, 0)):
        gM = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(theta=0.5, precision=R.FP64)))
        oM = oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec, amg=oracle.AmgParams(theta=0.5)))
        _hier_compare(gM.amg(0), oM.amg(0))
        if kind == 3:
            _hier_compare(gM.amg(1), oM.amg(1))


@pytest.mark.parametrize("prec", ["FP32", "FP64"])
def test_gmres_3d_matches_oracle(R, oracle, inputs, prec):
    p = inputs.config_layered_3d(n=16, layers=4)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    b = -Fo
    x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
    M = R.Precond(J, R.PrecParams(kind=R.CPR1, amg=R.AmgParams(theta=0.5, precision=getattr(R, prec))))
    st = R.gmres_solve(J, M, _dev(b), x, R.GmresParams(rtol=1e-8, maxit=500))
    assert st.status == R.RS_OK, st
    xg = x.cpu().numpy()
    res = b - oracle.bsr2_spmv(rp, col, Jo, xg)
    assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(b)
    xo, sto, _, _ = oracle.fgmres(rp, col, Jo, b, oracle.Precond(rp, col, Jo, oracle.PrecParams(
        kind=1, decouple=2, amg=oracle.AmgParams(theta=0.5))), maxit=500)
    assert sto == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6


@pytest.mark.parametrize("cc", [0, 64, 128])
def test_coarse_chunk_option_matches_oracle(R, oracle, inputs, cc):
    """The coarse-level chunk of the hybrid smoother (0: `chunk` on every
    level): same colourings as the oracle, and the FP64 V-cycle within
    1e-10, for scalar and point AMG."""
    p = inputs.config_lognormal_2d(1e3, n=40)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    jrp, jc, jv = oracle.scalar_from_bsr2(rp, col, Jo).arrays()
    for arp, ac, av, nf in ((*inputs.poisson_2d(50), 1), (jrp, jc, jv, 2)):
        oh = oracle.Amg(oracle.Csr.from_arrays(arp, ac, av), oracle.AmgParams(num_functions=nf, chunk_coarse=cc))
        gh = R.Amg.setup(R.Csr(arp, ac, av), R.AmgParams(num_functions=nf, chunk_coarse=cc, precision=R.FP64))
        _hier_compare(gh, oh)
        b = inputs.rhs_vector(arp.size - 1, 2)
        x = torch.empty(arp.size - 1, dtype=torch.float64, device="cuda")
        gh.apply(_dev(b), x)
        xo = oh.vcycle(b)
        np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=1e-10, atol=1e-11 * np.abs(xo).max())

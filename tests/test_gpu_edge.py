"""Edge cases of the GPU path through the C-ABI, against the oracle or exact
solves: an empty system, a single cell, a one-row strip (1D flow), a ragged
batch with a single-cell member, and a one-level hierarchy (the V-cycle is
then the dense coarse solve, so FGMRES converges in one iteration)."""
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_empty_system(R):
    J = R.Bsr2.from_host(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    x = torch.zeros(0, dtype=torch.float64, device="cuda")
    y = torch.zeros(0, dtype=torch.float64, device="cuda")
    R.bsr2_spmv(J, x, y)
    for kind in (R.AMG_J, R.CPR1, R.CPR2, R.BF):
        M = R.Precond(J, R.PrecParams(kind=kind, decouple=0))
        M.apply(x, y)
        st = R.gmres_solve(J, M, x, y, R.GmresParams())
        assert st.status == R.RS_OK and st.iterations == 0 and st.converged == 1
        M.close()
    H = R.Amg.setup(R.Csr(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)), R.AmgParams())
    assert H.nlevels == 1 and H.level_info(0)[0] == 0
    H.apply(x, y)
    torch.cuda.synchronize()


@pytest.mark.parametrize("shape", [(1, 1), (300, 1), (1, 150)])
@pytest.mark.parametrize("kind,dec", [(0, 0), (1, 2), (3, 0)])
def test_tiny_and_strip_grids_match_dense_solve(R, oracle, inputs, shape, kind, dec):
    p = inputs.homogeneous(*shape).with_(pc_model=2, pc_pd=5e3)
    u, uo = inputs.front_state(p)
    dp = R.DeviceProblems(p)
    J = R.Bsr2.pattern(dp)
    F = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(u), _dev(uo), inputs.DAY, J, F)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=1e-10, atol=1e-12 * np.abs(Fo).max())
    x = torch.zeros_like(F)
    for prec in (R.FP32, R.FP64):
        x.zero_()
        M = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=prec)))
        st = R.gmres_solve(J, M, -F, x, R.GmresParams(maxit=200))
        assert st.status == R.RS_OK, (shape, kind, prec, st)
        A = oracle.bsr2_to_scipy(rp, col, Jo).toarray()
        xe = np.linalg.solve(A, -Fo)
        np.testing.assert_allclose(x.cpu().numpy(), xe, rtol=1e-6, atol=1e-6 * np.abs(xe).max())
        M.close()


def test_ragged_batch_with_single_cell_member(R, oracle, inputs):
    probs = [inputs.homogeneous(1, 1).with_(pc_model=2, pc_pd=5e3), inputs.config_lognormal_2d(1e4, n=40, member=3),
             inputs.homogeneous(7, 1).with_(pc_model=2, pc_pd=5e3), inputs.homogeneous(3, 5).with_(pc_model=2, pc_pd=5e3)]
    states = [inputs.front_state(p) for p in probs]
    dp = R.DeviceProblems(probs)
    J = R.Bsr2.pattern(dp)
    F = torch.empty(2 * dp.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(np.concatenate([s[0] for s in states])),
                        _dev(np.concatenate([s[1] for s in states])), inputs.DAY, J, F)
    for kind, dec in ((0, 0), (1, 2), (3, 0)):
        x = torch.zeros_like(F)
        M = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=R.FP32)))
        st = R.gmres_solve(J, M, -F, x, R.GmresParams(maxit=300))
        assert st.status == R.RS_OK and st.converged == len(probs), (kind, st)
        xg = x.cpu().numpy()
        off = dp.cell_off
        for k, p in enumerate(probs):
            Fo, Jo, (rp, col) = oracle.assemble(p, states[k][0], states[k][1], inputs.DAY)
            res = -Fo - oracle.bsr2_spmv(rp, col, Jo, xg[2 * off[k]:2 * off[k + 1]])
            assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(Fo), (kind, k)
        M.close()


def test_one_level_hierarchy_is_exact(R, oracle, inputs):
    """coarse_n above the system size: no coarsening, the V-cycle is the dense
    FP64 coarse solve, and FGMRES preconditioned by it converges at once."""
    p = inputs.config_lognormal_2d(1e3, n=12)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    App = oracle.bsr2_part(rp, col, Jo, 0, 0)
    arp, ac, av = App.arrays()
    H = R.Amg.setup(R.Csr(arp, ac, av), R.AmgParams(coarse_n=10 ** 6, precision=R.FP64))
    assert H.nlevels == 1
    b = inputs.rhs_vector(p.ncell, 4)
    x = torch.empty(p.ncell, dtype=torch.float64, device="cuda")
    H.apply(_dev(b), x)
    xe = np.linalg.solve(App.scipy().toarray(), b)
    np.testing.assert_allclose(x.cpu().numpy(), xe, rtol=1e-10, atol=1e-12 * np.abs(xe).max())
    J = R.Bsr2.from_host(rp, col, Jo)
    M = R.Precond(J, R.PrecParams(kind=R.AMG_J, amg=R.AmgParams(coarse_n=10 ** 6, precision=R.FP64)))
    xj = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
    st = R.gmres_solve(J, M, _dev(-Fo), xj, R.GmresParams())
    assert st.status == R.RS_OK and st.iterations == 1


def test_fp32_hierarchy_beyond_range_is_rejected(R, oracle, inputs):
    """The unknown-agnostic scalar AMG on the 256^2 Jacobian builds coarse
    values beyond the FP32 range (the oracle pins that); an FP32 hierarchy is
    refused at set-up with a clear error, the FP64 one is built."""
    p = inputs.config_lognormal_2d(0.0, n=256)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    with pytest.raises(R.RsError, match="FP32 range"):
        R.Precond(J, R.PrecParams(kind=R.AMG_J_SCALAR, amg=R.AmgParams(precision=R.FP32)))
    M = R.Precond(J, R.PrecParams(kind=R.AMG_J_SCALAR, amg=R.AmgParams(precision=R.FP64)))
    M.close()


@pytest.mark.parametrize("wells", [dict(well_in=-2), dict(well_in=10 ** 6), dict(well_out=0),
                                   dict(well_out=10 ** 6)])
def test_bad_well_cells_are_rejected(R, inputs, wells):
    """A well cell outside the grid, or an outlet cell that is not on the
    x = L face, is refused before any launch."""
    good = inputs.homogeneous(6, 4).with_(pc_model=2, pc_pd=5e3)
    u, uo = inputs.front_state(good)
    J = R.Bsr2.pattern(R.DeviceProblems(good))
    F = torch.empty(2 * good.ncell, dtype=torch.float64, device="cuda")
    dp = R.DeviceProblems(good.with_(**wells))
    with pytest.raises(R.RsError, match="well"):
        R.Bsr2.pattern(dp)
    with pytest.raises(R.RsError, match="well"):
        R.jacobian_assemble(dp, _dev(u), _dev(uo), inputs.DAY, J, F)


def test_two_cell_fluxes_hand_values(R, two_cell_cases):
    """GPU assembly on the hand-derived two-cell cases (harmonic face
    permeability, per-phase upwinding in both directions, the tie rule in
    the Jacobian, a z face in 3D): the same values the oracle is pinned to."""
    cases, dt = two_cell_cases
    for c, p, u in cases:
        dp = R.DeviceProblems(p)
        J = R.Bsr2.pattern(dp)
        F = torch.empty(4, dtype=torch.float64, device="cuda")
        ud = _dev(u)
        R.jacobian_assemble(dp, ud, ud, dt, J, F)
        torch.cuda.synchronize()
        Fh = F.cpu().numpy()
        np.testing.assert_allclose(Fh[:2], c["F0"], rtol=1e-12, atol=1e-20, err_msg=c["name"])
        if "J00_pw_pw" in c:
            rp = J.row_ptr.cpu().numpy()
            assert list(J.col.cpu().numpy()[rp[0]:rp[1]]) == [0, 1]
            val = J.val.cpu().numpy().reshape(-1, 2, 2)
            np.testing.assert_allclose(val[rp[0], 0, 0], c["J00_pw_pw"], rtol=1e-12, err_msg=c["name"])
            np.testing.assert_allclose(val[rp[0] + 1, 0, 0], c["J01_pw_pw"], rtol=1e-12, err_msg=c["name"])


def test_capped_wait_reported_and_cleared(R, inputs):
    """A smoother CTA that gives up waiting for its staging copies raises a
    device flag. Here the flag is raised from the host (no kernel is made to
    time out): gmres_solve reports RS_ETIMEOUT and clears it, so the next
    solve succeeds; rs_wait_status reports it after the asynchronous
    precond_apply; newton_step returns the error with its statistics
    filled in for the iteration that met it."""
    import ctypes
    p = inputs.config_small_2d()
    u, uo = inputs.front_state(p)
    dp = R.DeviceProblems(p)
    J = R.Bsr2.pattern(dp)
    F = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(u), _dev(uo), inputs.DAY, J, F)
    b = -F
    M = R.Precond(J, R.PrecParams(kind=R.CPR1))
    assert R.wait_status() == R.RS_OK
    R.raise_wait_flag()
    with pytest.raises(R.RsError, match="wait limit"):
        R.gmres_solve(J, M, b, torch.zeros_like(b), R.GmresParams(rtol=1e-8))
    x = torch.zeros_like(b)
    st = R.gmres_solve(J, M, b, x, R.GmresParams(rtol=1e-8))
    assert st.status == R.RS_OK
    z = torch.empty_like(b)
    M.apply(b, z)
    assert R.wait_status() == R.RS_OK
    R.raise_wait_flag()
    M.apply(b, z)
    assert R.wait_status() == R.RS_ETIMEOUT
    assert R.wait_status() == R.RS_OK
    M.close()
    # newton_step through the C-ABI directly, to read its statistics
    L = R.lib()
    prm = R.NewtonParams(prec=R.PrecParams(kind=R.CPR1))
    stc = R.NewtonStatsC()
    ud = _dev(u)
    R.raise_wait_flag()
    rc = L.newton_step(dp.c, len(dp), R._ptr(ud), R._ptr(_dev(uo)), inputs.DAY, ctypes.byref(prm.c()),
                       ctypes.byref(stc), R._stream())
    assert rc == R.RS_ETIMEOUT
    assert stc.newton_its == 1 and stc.linear_its > 0 and stc.fnorm > 0
    assert R.wait_status() == R.RS_OK

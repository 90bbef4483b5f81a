"""ILU(0) on the GPU (the first stage P1 of CPR, Sec. 3.3) against the oracle.

The level-scheduled factorisation and triangular solves run each cell's two
rows in the sequential algorithm's operation order without FMA contraction,
so factors and solves are compared bit for bit: 2D and 3D Jacobians, a
batch of stacked grids, and 3D grids wide enough for clusters of 2, 4 and 8
CTAs. The level schedule of a Cartesian grid in lexicographic order is its
set of anti-diagonals (nx + ny - 1 levels in 2D, nx + ny + nz - 2 in 3D).
CPR with P1 = ILU(0) applies and solves like the oracle's; a pattern that is
not structurally symmetric, or lacks a diagonal block, is refused.
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _jacobian(oracle, inputs, p, seed=0):
    u, uo = inputs.front_state(p)
    u = inputs.jitter(u, seed)
    F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    return F, J, rp, col


def _grids(inputs):
    rng = np.random.default_rng(11)
    k3 = np.exp(rng.normal(np.log(1e-12), 1.0, 9 * 6 * 5))
    return [inputs.config_gravity_2d(20, 2), inputs.config_lognormal_2d(1e4, n=48),
            inputs.Problem(dim=3, nx=9, ny=6, nz=5, kx=k3, ky=k3 * 0.5, kz=k3 * 0.1, pc_model=2, pc_pd=5e3),
            inputs.homogeneous(37, 1).with_(pc_model=2, pc_pd=5e3)]


@pytest.mark.parametrize("case", range(4))
def test_ilu0_factors_and_solve_bit_exact(R, oracle, inputs, case):
    p = _grids(inputs)[case]
    F, J, rp, col = _jacobian(oracle, inputs, p, case)
    Jd = R.Bsr2.from_host(rp, col, J)
    f = R.Ilu0(Jd)
    nlev, maxw, ctas = f.info()
    if p.dim == 2:
        assert nlev == p.nx + p.ny - 1 and maxw == min(p.nx, p.ny)
    else:
        assert nlev == p.nx + p.ny + p.nz - 2
    assert ctas == 1
    lu = oracle.ilu0(rp, col, J)
    np.testing.assert_array_equal(f.factors().cpu().numpy().reshape(-1, 2, 2), lu)
    b = inputs.rhs_vector(2 * p.ncell, case)
    x = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    f.apply(_dev(b), x)
    np.testing.assert_array_equal(x.cpu().numpy(), oracle.ilu0_solve(rp, col, lu, b))
    f.close()


def test_ilu0_batch_of_grids_bit_exact(R, oracle, inputs):
    probs = _grids(inputs)
    parts = [_jacobian(oracle, inputs, p, k) for k, p in enumerate(probs)]
    rps, cols, Js, off = [], [], [], [0]
    for F, J, rp, col in parts:
        rps.append(rp[:-1] + sum(len(c) for c in cols))
        cols.append(col + off[-1])
        Js.append(J)
        off.append(off[-1] + rp.size - 1)
    rp = np.concatenate(rps + [[sum(len(c) for c in cols)]]).astype(np.int32)
    col = np.concatenate(cols).astype(np.int32)
    J = np.concatenate(Js)
    f = R.Ilu0(R.Bsr2.from_host(rp, col, J, seg_off=np.asarray(off, np.int32)))
    nlev, maxw, _ = f.info()
    assert nlev == max(p.nx + p.ny + p.nz - 2 for p in probs)
    lu = f.factors().cpu().numpy().reshape(-1, 2, 2)
    for k, (F, Jk, rpk, colk) in enumerate(parts):
        b0, b1 = rp[off[k]], rp[off[k + 1]]
        np.testing.assert_array_equal(lu[b0:b1], oracle.ilu0(rpk, colk, Jk))


@pytest.mark.parametrize("n,ctas", [(24, 1), (40, 2), (56, 4), (80, 8)])
def test_ilu0_wide_levels_use_clusters(R, oracle, inputs, n, ctas):
    """3D grids whose widest level needs 1, 2, 4 and 8 CTAs of 1024 threads
    (80^3: 512,000 cells, widest anti-diagonal plane 4,800 cells)."""
    k = np.full(n ** 3, 1e-12)
    p = inputs.Problem(dim=3, nx=n, ny=n, nz=n, kx=k, ky=k, kz=k * 0.1, pc_model=2, pc_pd=5e3)
    F, J, rp, col = _jacobian(oracle, inputs, p, 3)
    f = R.Ilu0(R.Bsr2.from_host(rp, col, J))
    nlev, maxw, c = f.info()
    assert nlev == 3 * n - 2 and c == ctas, (nlev, maxw, c)
    lu = oracle.ilu0(rp, col, J)
    np.testing.assert_array_equal(f.factors().cpu().numpy().reshape(-1, 2, 2), lu)
    b = inputs.rhs_vector(2 * p.ncell, 7)
    x = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    f.apply(_dev(b), x)
    np.testing.assert_array_equal(x.cpu().numpy(), oracle.ilu0_solve(rp, col, lu, b))


def test_ilu0_rejects_bad_patterns(R, inputs, oracle):
    p = inputs.homogeneous(4, 3).with_(pc_model=2, pc_pd=5e3)
    F, J, rp, col = _jacobian(oracle, inputs, p)
    # drop block (1, 0) but keep (0, 1): not structurally symmetric
    k10 = rp[1]
    assert col[k10] == 0
    rp2 = rp.copy()
    rp2[2:] -= 1
    col2 = np.delete(col, k10)
    J2 = np.delete(J, k10, axis=0)
    with pytest.raises(R.RsError, match="symmetric"):
        R.Ilu0(R.Bsr2.from_host(rp2, col2, J2))
    # drop the diagonal block of row 0
    kd = rp[0]
    assert col[kd] == 0
    rp3 = rp.copy()
    rp3[1:] -= 1
    col3 = np.delete(col, kd)
    J3 = np.delete(J, kd, axis=0)
    with pytest.raises(R.RsError, match="diagonal"):
        R.Ilu0(R.Bsr2.from_host(rp3, col3, J3))


@pytest.mark.parametrize("kind,dec", [(1, 0), (1, 1), (1, 2), (2, 2)])
def test_cpr_with_ilu0_matches_oracle(R, oracle, inputs, kind, dec):
    p = inputs.config_gravity_2d(24, 2)
    F, J, rp, col = _jacobian(oracle, inputs, p, 5)
    Jd = R.Bsr2.from_host(rp, col, J)
    prm = dict(kind=kind, decouple=dec, p1=1)
    M = R.Precond(Jd, R.PrecParams(**prm, amg=R.AmgParams(precision=R.FP64)))
    Mo = oracle.Precond(rp, col, J, oracle.PrecParams(**prm))
    r = inputs.rhs_vector(2 * p.ncell, 3)
    z = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    for _ in range(3):                      # eager apply, then the recorded graph
        M.apply(_dev(r), z)
        zo = Mo.apply(r)
        np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-10, atol=1e-10 * np.abs(zo).max())
    x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
    st = R.gmres_solve(Jd, M, _dev(-F), x, R.GmresParams(maxit=400))
    xo, sto, ito, _ = oracle.fgmres(rp, col, J, -F, Mo, maxit=400)
    assert st.status == R.RS_OK and sto == 0
    assert abs(st.iterations - ito) <= 1
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=1e-6, atol=1e-6 * np.abs(xo).max())
    M.close()


@pytest.mark.parametrize("case", [0, 1, 2])
def test_ilu0_fp32_solves_close_to_fp64(R, oracle, inputs, case):
    """FP32 solves (the factors rounded once, FP32 sweeps): within 1e-4 of
    the oracle's FP64 solve, relative in the 2-norm; FP32 rounding amplified
    by the triangular factors' conditioning."""
    p = _grids(inputs)[case]
    F, J, rp, col = _jacobian(oracle, inputs, p, case)
    f = R.Ilu0(R.Bsr2.from_host(rp, col, J), R.FP32)
    b = inputs.rhs_vector(2 * p.ncell, case)
    x = torch.empty(2 * p.ncell, dtype=torch.float64, device="cuda")
    f.apply(_dev(b), x)
    xo = oracle.ilu0_solve(rp, col, oracle.ilu0(rp, col, J), b)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-4 * np.linalg.norm(xo)


@pytest.mark.parametrize("kind", [1, 2])
def test_cpr_ilu0_fp32_converges_like_fp64(R, oracle, inputs, kind):
    p = inputs.config_gravity_2d(40, 1)
    F, J, rp, col = _jacobian(oracle, inputs, p, 2)
    Jd = R.Bsr2.from_host(rp, col, J)
    its = {}
    for prec in (R.FP32, R.FP64):
        M = R.Precond(Jd, R.PrecParams(kind=kind, decouple=2, p1=1, amg=R.AmgParams(precision=prec)))
        x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
        st = R.gmres_solve(Jd, M, _dev(-F), x, R.GmresParams(maxit=600))
        assert st.status == R.RS_OK
        res = -F - oracle.bsr2_spmv(rp, col, J, x.cpu().numpy())
        assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(F)
        its[prec] = st.iterations
        M.close()
    assert its[R.FP32] <= 1.15 * its[R.FP64] + 2, its

"""Aggressive coarsening (two-stage form) on the GPU against the oracle:
hierarchies bit-exact (splittings, merged interpolation, operators,
colourings) for scalar and systems (point) AMG with one and two aggressive
levels, the FP64 V-cycle within 1e-10, and FGMRES with the point AMG
converging like the oracle's."""
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


def _compare(gh, oh):
    assert gh.sizes() == oh.sizes()
    for l in range(oh.nlevels):
        g = gh.level(l)
        for got, ref in zip(g["A"], oh.A(l).arrays()):
            np.testing.assert_array_equal(got, ref)
        if l + 1 < oh.nlevels:
            np.testing.assert_array_equal(g["cf"], oh.cf(l))
            for got, ref in zip(g["P"], oh.P(l).arrays()):
                np.testing.assert_array_equal(got, ref)
            col, nc = oh.colours(l)
            assert g["ncolours"] == nc
            np.testing.assert_array_equal(g["colour"], col)


def _systems(oracle, inputs):
    rp, c, v = inputs.poisson_2d(60)
    p = inputs.config_lognormal_2d(1e4, n=40)
    u, uo = inputs.front_state(p)
    Fo, Jo, (brp, bcol) = oracle.assemble(p, u, uo, inputs.DAY)
    jrp, jc, jv = oracle.scalar_from_bsr2(brp, bcol, Jo).arrays()
    return {"poisson": (rp, c, v, 1), "J_point": (jrp, jc, jv, 2)}


@pytest.mark.parametrize("agg", [1, 2])
@pytest.mark.parametrize("which", ["poisson", "J_point"])
def test_aggressive_hierarchy_bit_exact(R, oracle, inputs, agg, which):
    rp, c, v, nf = _systems(oracle, inputs)[which]
    oh = oracle.Amg(oracle.Csr.from_arrays(rp, c, v), oracle.AmgParams(num_functions=nf, agg_levels=agg, coarse_n=40))
    gh = R.Amg.setup(R.Csr(rp, c, v), R.AmgParams(num_functions=nf, agg_levels=agg, coarse_n=40, precision=R.FP64))
    _compare(gh, oh)
    b = inputs.rhs_vector(rp.size - 1, 4)
    x = torch.empty(rp.size - 1, dtype=torch.float64, device="cuda")
    gh.apply(_dev(b), x)
    xo = oh.vcycle(b)
    np.testing.assert_allclose(x.cpu().numpy(), xo, rtol=1e-10, atol=1e-11 * np.abs(xo).max())


def test_aggressive_point_amg_fgmres_matches_oracle(R, oracle, inputs):
    p = inputs.config_lognormal_2d(1e3, n=48)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    for prec in (R.FP64, R.FP32):
        M = R.Precond(J, R.PrecParams(kind=R.AMG_J, decouple=0, amg=R.AmgParams(agg_levels=1, precision=prec)))
        x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
        st = R.gmres_solve(J, M, _dev(-Fo), x, R.GmresParams(maxit=400))
        Mo = oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=0, decouple=0, amg=oracle.AmgParams(agg_levels=1)))
        xo, sto, ito, _ = oracle.fgmres(rp, col, Jo, -Fo, Mo, maxit=400)
        assert st.status == R.RS_OK and sto == 0
        if prec == R.FP64:
            assert abs(st.iterations - ito) <= 1
        res = -Fo - oracle.bsr2_spmv(rp, col, Jo, x.cpu().numpy())
        assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(Fo)
        M.close()

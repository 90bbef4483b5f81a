"""The coarse tail (the levels below `tail_rows` rows run as one cluster
launch) computes the same V-cycle as one launch per kernel and level: FP64
within 1e-10 of the oracle and within 1e-11 of the per-level path, FP32
within 1e-5 of the oracle, for scalar AMG (Poisson, the CPR pressure block,
the SIMPLE Schur complement) and systems (point) AMG on J, including a
hierarchy whose every level below the finest lies in the tail; FGMRES with
the tail matches the
oracle's iteration counts and solutions."""
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


def _matrices(oracle, inputs):
    p = inputs.config_lognormal_2d(1e3, n=64)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    App = oracle.bsr2_part(rp, col, oracle.decouple_abf(rp, col, Jo), 0, 0)
    St = oracle.simple_schur(*[oracle.bsr2_part(rp, col, Jo, r, c) for r, c in ((0, 0), (0, 1), (1, 0), (1, 1))])
    return {"poisson": (*inputs.poisson_2d(90), 1), "poisson_small": (*inputs.poisson_2d(20), 1),
            "App": (*App.arrays(), 1), "Stilde": (*St.arrays(), 1),
            "J_point": (*oracle.scalar_from_bsr2(rp, col, Jo).arrays(), 2)}


@pytest.mark.parametrize("which", ["poisson", "poisson_small", "App", "Stilde", "J_point"])
def test_tail_vcycle_matches_oracle_and_per_level_path(R, oracle, inputs, which):
    rp, c, v, nf = _matrices(oracle, inputs)[which]
    oh = oracle.Amg(oracle.Csr.from_arrays(rp, c, v), oracle.AmgParams(num_functions=nf))
    n = rp.size - 1
    b = inputs.rhs_vector(n, 3)
    xo = oh.vcycle(b)
    out = {}
    for prec in (R.FP64, R.FP32):
        for tail in (0, 4096):
            gh = R.Amg.setup(R.Csr(rp, c, v), R.AmgParams(num_functions=nf, precision=prec, tail_rows=tail))
            t = gh.tail_level()
            if tail:
                assert 0 <= t <= gh.nlevels - 2, (which, t, gh.sizes())
                assert all(sz <= 4096 for sz in gh.sizes()[t:])
                if which == "poisson_small":
                    assert t == 1      # level 0's 512-row chunk is too long for a warp; the rest is tail
            else:
                assert t == -1
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            gh.apply(_dev(b), x)
            gh.apply(_dev(b), x)            # the same result on a second cycle
            out[prec, tail] = x.cpu().numpy()
    scale = np.abs(xo).max()
    np.testing.assert_allclose(out[R.FP64, 4096], xo, rtol=1e-10, atol=1e-11 * scale)
    np.testing.assert_allclose(out[R.FP64, 4096], out[R.FP64, 0], rtol=1e-11, atol=1e-12 * scale)
    assert np.linalg.norm(out[R.FP32, 4096] - xo) <= 1e-5 * np.linalg.norm(xo)


@pytest.mark.parametrize("kind,dec", [(0, 0), (1, 2), (2, 2), (3, 0)])
def test_tail_fgmres_matches_oracle(R, oracle, inputs, kind, dec):
    p = inputs.config_lognormal_2d(1e3, n=64)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    J = R.Bsr2.from_host(rp, col, Jo)
    xo, sto, ito, _ = oracle.fgmres(rp, col, Jo, -Fo, oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec)),
                                    maxit=400)
    assert sto == 0
    for prec in (R.FP64, R.FP32):
        M = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=prec, tail_rows=4096)))
        assert M.amg(0).tail_level() >= 0
        x = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
        st = R.gmres_solve(J, M, _dev(-Fo), x, R.GmresParams(maxit=400))
        assert st.status == R.RS_OK
        if prec == R.FP64:
            assert abs(st.iterations - ito) <= 1, (st.iterations, ito)
        xg = x.cpu().numpy()
        assert np.linalg.norm(-Fo - oracle.bsr2_spmv(rp, col, Jo, xg)) <= 1.0001e-8 * np.linalg.norm(Fo)
        assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
        M.close()

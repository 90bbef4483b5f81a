"""Full-size workloads on the GPU, checked by the oracle.

* 256x256 log-normal (the benchmark workload): every black-box AMG (point
  method) and CPR solve and the BF solves that converge, FP32 and FP64
  V-cycles, against the oracle's solution (1e-6) and residual (1e-8).
* 128^3 layered grid: the first Jacobian solved with FP32 and FP64
  hierarchies (true residual by the oracle, FP32-vs-FP64 difference), and ten
  backward-Euler time steps whose every result the oracle's residual accepts.
* 256^3 channelised grid: one Newton step each with CPR and block
  factorisation, accepted by the oracle's residual.
* 96-member ensemble (sides 64..512): one batched CPR solve; every member's
  true residual recomputed by the oracle.
Too large for an element-by-element oracle solve are checked through
properties that hold at any size (the oracle's residual of the GPU result).
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


@pytest.mark.parametrize("pc", [0.0, 1e3, 1e4, 1e5])
def test_lognormal_256_solves_match_oracle(R, oracle, inputs, pc):
    p = inputs.config_lognormal_2d(pc, n=256)
    u, uo = inputs.front_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    b = -Fo
    J = R.Bsr2.from_host(rp, col, Jo)
    kinds = [(0, 0), (1, 2)] + ([(3, 0)] if pc <= 1e3 else [])
    for kind, dec in kinds:
        xo, sto, ito, _ = oracle.fgmres(rp, col, Jo, b, oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec)),
                                        maxit=400)
        assert sto == 0
        for prec in (R.FP32, R.FP64):
            x = torch.zeros_like(_dev(b))
            M = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=prec)))
            st = R.gmres_solve(J, M, _dev(b), x, R.GmresParams(maxit=400))
            assert st.status == R.RS_OK, (kind, prec, st)
            xg = x.cpu().numpy()
            res = b - oracle.bsr2_spmv(rp, col, Jo, xg)
            assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(b)
            assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6


def test_layered_128_first_jacobian_fp32_vs_fp64(R, oracle, inputs):
    """First Jacobian of the first time step, solved with an FP32 and an FP64
    V-cycle inside FP64 FGMRES: both meet 1e-8 by the oracle's residual and
    agree with each other within the solution tolerance."""
    p = inputs.config_layered_3d(128)
    u0 = inputs.initial_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u0, u0, inputs.DAY)
    b = -Fo
    J = R.Bsr2.from_host(rp, col, Jo)
    xs = {}
    for prec in (R.FP32, R.FP64):
        x = torch.zeros_like(_dev(b))
        M = R.Precond(J, R.PrecParams(kind=R.CPR1, amg=R.AmgParams(theta=0.5, precision=prec)))
        st = R.gmres_solve(J, M, _dev(b), x, R.GmresParams(maxit=500))
        assert st.status == R.RS_OK, st
        xs[prec] = x.cpu().numpy()
        res = b - oracle.bsr2_spmv(rp, col, Jo, xs[prec])
        assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(b)
        M.close()
    d = np.linalg.norm(xs[R.FP32] - xs[R.FP64]) / np.linalg.norm(xs[R.FP64])
    assert d <= 1e-6, d


def test_layered_128_ten_time_steps(R, oracle, inputs):
    """Ten backward-Euler steps of one day on the 128^3 layered grid, Newton
    with CPR FGMRES, once with FP32 and once with FP64 V-cycles: after every
    step the oracle's scaled residual of the GPU state meets the Newton
    tolerance, and the two sequences agree."""
    p = inputs.config_layered_3d(128)
    rp, col = oracle.bsr2_pattern(p)
    dp = R.DeviceProblems(p)
    seq = {}
    for prec in (R.FP32, R.FP64):
        prm = R.NewtonParams(prec=R.PrecParams(kind=R.CPR1, amg=R.AmgParams(theta=0.5, precision=prec)))
        u = _dev(inputs.initial_state(p))
        states = []
        for step in range(10):
            u_old = u.clone()
            rc, st = R.newton_step(dp, u, u_old, inputs.DAY, prm)
            assert rc == R.RS_OK, (prec, step, st)
            uh, uoh = u.cpu().numpy(), u_old.cpu().numpy()
            F, _, _ = oracle.assemble(p, uh, uoh, inputs.DAY, pattern=(rp, col), jacobian=False)
            assert oracle.scaled_fnorm(p, F, inputs.DAY) <= 1e-6, (prec, step)
            states.append(uh)
        seq[prec] = states
    for a, b in zip(seq[R.FP32], seq[R.FP64]):
        np.testing.assert_allclose(a[0::2], b[0::2], rtol=1e-6)
        np.testing.assert_allclose(a[1::2], b[1::2], atol=1e-6)
    # the injected water has moved the saturation
    assert np.abs(seq[R.FP64][-1][1::2] - inputs.initial_state(p)[1::2]).max() > 1e-3


@pytest.mark.parametrize("kind", ["CPR1", "BF"])
def test_channel_256_newton_step(R, oracle, inputs, kind):
    """The 256^3 channelised grid (33.5M unknowns): one backward-Euler Newton
    step with FP32 V-cycles; the oracle's scaled residual of the result meets
    the Newton tolerance."""
    p = inputs.config_channel_3d(256)
    u0 = inputs.initial_state(p)
    dp = R.DeviceProblems(p)
    u = _dev(u0)
    prm = R.NewtonParams(prec=R.PrecParams(kind=getattr(R, kind), amg=R.AmgParams(theta=0.5, precision=R.FP32)))
    rc, st = R.newton_step(dp, u, _dev(u0), inputs.DAY, prm)
    assert rc == R.RS_OK, st
    F, _, _ = oracle.assemble(p, u.cpu().numpy(), u0, inputs.DAY, jacobian=False)
    assert oracle.scaled_fnorm(p, F, inputs.DAY) <= 1e-6


def test_ensemble_96_batched_solve(R, oracle, inputs):
    probs = inputs.config_ensemble()
    assert len(probs) == 96
    states = [inputs.front_state(p) for p in probs]
    dp = R.DeviceProblems(probs)
    J = R.Bsr2.pattern(dp)
    F = torch.empty(2 * dp.ncell, dtype=torch.float64, device="cuda")
    R.jacobian_assemble(dp, _dev(np.concatenate([s[0] for s in states])),
                        _dev(np.concatenate([s[1] for s in states])), inputs.DAY, J, F)
    b = -F
    x = torch.zeros_like(b)
    M = R.Precond(J, R.PrecParams(kind=R.CPR1, amg=R.AmgParams(precision=R.FP32)))
    st = R.gmres_solve(J, M, b, x, R.GmresParams(maxit=600))
    assert st.status == R.RS_OK and st.converged == 96, st
    xg = x.cpu().numpy()
    off = dp.cell_off
    for k, p in enumerate(probs):
        Fo, Jo, (rp, col) = oracle.assemble(p, states[k][0], states[k][1], inputs.DAY)
        xk = xg[2 * off[k]:2 * off[k + 1]]
        res = -Fo - oracle.bsr2_spmv(rp, col, Jo, xk)
        assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(Fo), k
        if p.nx == 64 and k < 40:
            xo, sto, _, _ = oracle.fgmres(rp, col, Jo, -Fo, oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=1, decouple=2)))
            assert np.linalg.norm(xk - xo) / np.linalg.norm(xo) <= 1e-6

"""Full-size workloads on the GPU, checked by the oracle.

* 256x256 log-normal: every black-box AMG (point method) and CPR solve,
  block factorisation with lAIR hierarchies at every capillary scale and
  with Galerkin hierarchies where they converge, FP32 and FP64 V-cycles,
  against the oracle's solution (1e-6) and residual (1e-8).
* 128^3 layered grid: the first Jacobian solved with CPR-AMG and block
  factorisation, FP32 and FP64 V-cycles, against the oracle's solution
  (1e-6) and residual (1e-8); ten backward-Euler time steps with each
  preconditioner in both precisions, every result accepted by the oracle's
  residual.
* 256^3 channelised grid: the first Jacobian solved with both
  preconditioners (the oracle's residual), and the five-step Newton
  sequence with each, the final state accepted by the oracle's residual.
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
    # block factorisation with the paper's Galerkin hierarchies where they
    # converge, and with lAIR (restriction 3) at every capillary scale
    kinds = [(0, 0, 0), (1, 2, 0), (3, 0, 3)] + ([(3, 0, 0)] if pc <= 1e3 else [])
    for kind, dec, restr in kinds:
        Mo = oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=kind, decouple=dec,
                                                           amg=oracle.AmgParams(restriction=restr)))
        xo, sto, ito, _ = oracle.fgmres(rp, col, Jo, b, Mo, maxit=400)
        assert sto == 0
        for prec in (R.FP32, R.FP64):
            x = torch.zeros_like(_dev(b))
            M = R.Precond(J, R.PrecParams(kind=kind, decouple=dec, amg=R.AmgParams(precision=prec, restriction=restr)))
            st = R.gmres_solve(J, M, _dev(b), x, R.GmresParams(maxit=400))
            assert st.status == R.RS_OK, (kind, prec, st)
            xg = x.cpu().numpy()
            res = b - oracle.bsr2_spmv(rp, col, Jo, xg)
            assert np.linalg.norm(res) <= 1.0001e-8 * np.linalg.norm(b)
            assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-6


KIND_3D = {"CPR1": (1, 2), "BF": (3, 0)}     # kind, decoupling (quasi-IMPES for CPR)


@pytest.fixture(scope="module")
def layered128(oracle, inputs):
    p = inputs.config_layered_3d(128)
    u0 = inputs.initial_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u0, u0, inputs.DAY)
    return p, u0, Fo, Jo, rp, col


@pytest.mark.parametrize("kind", ["CPR1", "BF"])
def test_layered_128_first_jacobian_vs_oracle(R, oracle, inputs, layered128, kind):
    """The 128^3 layered grid's first Jacobian (first Newton iterate of the
    first one-day step) solved by the oracle (FP64 FGMRES, FP64 V-cycles) and
    on the GPU with FP32 and with FP64 V-cycles inside FP64 FGMRES: every GPU
    solution meets 1e-8 by the oracle's residual and lies within 1e-6 of the
    oracle's solution. Prints the per-solve error against the oracle."""
    p, u0, Fo, Jo, rp, col = layered128
    k, dec = KIND_3D[kind]
    b = -Fo
    Mo = oracle.Precond(rp, col, Jo, oracle.PrecParams(kind=k, decouple=dec, amg=oracle.AmgParams(theta=0.5)))
    xo, sto, ito, _ = oracle.fgmres(rp, col, Jo, b, Mo, maxit=300)
    assert sto == 0
    J = R.Bsr2.from_host(rp, col, Jo)
    for prec, pn in ((R.FP32, "FP32"), (R.FP64, "FP64")):
        x = torch.zeros_like(_dev(b))
        M = R.Precond(J, R.PrecParams(kind=k, decouple=dec, amg=R.AmgParams(theta=0.5, precision=prec)))
        st = R.gmres_solve(J, M, _dev(b), x, R.GmresParams(maxit=300))
        M.close()
        assert st.status == R.RS_OK, (kind, pn, st)
        xg = x.cpu().numpy()
        rel = np.linalg.norm(b - oracle.bsr2_spmv(rp, col, Jo, xg)) / np.linalg.norm(b)
        err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
        print(f"\nlayered128 first Jacobian {kind} {pn} V-cycle: GPU {st.iterations} iterations "
              f"(oracle {ito}), oracle residual {rel:.2e}, error vs oracle {err:.2e}")
        assert rel <= 1.0001e-8
        assert err <= 1e-6


@pytest.mark.parametrize("kind", ["CPR1", "BF"])
def test_layered_128_ten_time_steps(R, oracle, inputs, kind):
    """Ten backward-Euler steps of one day on the 128^3 layered grid, Newton
    with FGMRES preconditioned by CPR-AMG or block factorisation, once with
    FP32 and once with FP64 V-cycles: after every step the oracle's scaled
    residual of the GPU state meets the Newton tolerance, and the two
    sequences agree."""
    p = inputs.config_layered_3d(128)
    rp, col = oracle.bsr2_pattern(p)
    dp = R.DeviceProblems(p)
    k, dec = KIND_3D[kind]
    seq = {}
    for prec, pn in ((R.FP32, "FP32"), (R.FP64, "FP64")):
        prm = R.NewtonParams(prec=R.PrecParams(kind=k, decouple=dec, amg=R.AmgParams(theta=0.5, precision=prec)))
        u = _dev(inputs.initial_state(p))
        states = []
        for step in range(10):
            u_old = u.clone()
            rc, st = R.newton_step(dp, u, u_old, inputs.DAY, prm)
            assert rc == R.RS_OK, (kind, pn, step, st)
            uh, uoh = u.cpu().numpy(), u_old.cpu().numpy()
            F, _, _ = oracle.assemble(p, uh, uoh, inputs.DAY, pattern=(rp, col), jacobian=False)
            fn = oracle.scaled_fnorm(p, F, inputs.DAY)
            print(f"\nlayered128 {kind} {pn} step {step + 1}: NI {st['newton_its']} LI {st['linear_its']} "
                  f"oracle scaled residual {fn:.2e}")
            assert fn <= 1e-6, (kind, pn, step)
            states.append(uh)
        seq[prec] = states
    for a, b in zip(seq[R.FP32], seq[R.FP64]):
        np.testing.assert_allclose(a[0::2], b[0::2], rtol=1e-6)
        np.testing.assert_allclose(a[1::2], b[1::2], atol=1e-6)
    # the injected water has moved the saturation
    assert np.abs(seq[R.FP64][-1][1::2] - inputs.initial_state(p)[1::2]).max() > 1e-3


@pytest.fixture(scope="module")
def channel256(inputs):
    return inputs.config_channel_3d(256)


def test_channel_256_first_jacobian_oracle_residual(R, oracle, inputs, channel256):
    """The 256^3 channelised grid's first Jacobian (33.5M unknowns) solved on
    the GPU with CPR-AMG and block factorisation, FP32 V-cycles in FP64
    FGMRES: the oracle's residual of every solution meets 1e-8 (an oracle
    solve of this size is out of reach; its residual is the check that holds
    at any size). Prints the per-solve residuals."""
    p = channel256
    u0 = inputs.initial_state(p)
    Fo, Jo, (rp, col) = oracle.assemble(p, u0, u0, inputs.DAY)
    b = -Fo
    J = R.Bsr2.from_host(rp, col, Jo)
    bd = _dev(b)
    for kind, (k, dec) in KIND_3D.items():
        x = torch.zeros_like(bd)
        M = R.Precond(J, R.PrecParams(kind=k, decouple=dec, amg=R.AmgParams(theta=0.5, precision=R.FP32)))
        st = R.gmres_solve(J, M, bd, x, R.GmresParams(maxit=300))
        M.close()
        assert st.status == R.RS_OK, (kind, st)
        rel = np.linalg.norm(b - oracle.bsr2_spmv(rp, col, Jo, x.cpu().numpy())) / np.linalg.norm(b)
        print(f"\nchannel256 first Jacobian {kind} FP32 V-cycle: {st.iterations} iterations, "
              f"GPU residual {st.relres:.2e}, oracle residual {rel:.2e}")
        assert rel <= 1.0001e-8


@pytest.mark.parametrize("kind", ["CPR1", "BF"])
def test_channel_256_five_time_steps(R, oracle, inputs, channel256, kind):
    """The 256^3 channelised grid's full Newton sequence: five one-day
    backward-Euler steps with FP32 V-cycles; every step converges (the
    Newton tolerance on the GPU's residual) and the oracle's scaled residual
    of the final state meets the tolerance."""
    p = channel256
    u0 = inputs.initial_state(p)
    dp = R.DeviceProblems(p)
    k, dec = KIND_3D[kind]
    prm = R.NewtonParams(prec=R.PrecParams(kind=k, decouple=dec, amg=R.AmgParams(theta=0.5, precision=R.FP32)))
    u = _dev(u0)
    for step in range(5):
        u_old = u.clone()
        rc, st = R.newton_step(dp, u, u_old, inputs.DAY, prm)
        print(f"\nchannel256 {kind} FP32 step {step + 1}: NI {st['newton_its']} LI {st['linear_its']} "
              f"residual {st['fnorm']:.2e} set-up {st['setup_ms']:.0f} ms solve {st['solve_ms']:.0f} ms")
        assert rc == R.RS_OK, (kind, step, st)
    F, _, _ = oracle.assemble(p, u.cpu().numpy(), u_old.cpu().numpy(), inputs.DAY, jacobian=False)
    fn = oracle.scaled_fnorm(p, F, inputs.DAY)
    print(f"\nchannel256 {kind} after 5 steps: oracle scaled residual {fn:.2e}")
    assert fn <= 1e-6


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

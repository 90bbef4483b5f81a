"""Pins of the oracle's Krylov solver, the four preconditioners and Newton.

* FGMRES against dense LU (numpy) on small systems.
* Algorithms 1, 2, 3 equal their matrix forms (eqs. m_comb, m_add, m_bf)
  when the inner AMG solves are exact (single-level hierarchy = LU).
* Block factorisation with an exact Schur complement: (J M^{-1} - I)^2 = 0,
  so GMRES converges in at most two iterations (Sec. 3.4).
* Newton converges quadratically (Sec. 3).
"""
import numpy as np
import pytest
import scipy.sparse as sp


def _tiny(I, O, nx=4, ny=3, pc=2, seed=0):
    rng = np.random.default_rng(seed)
    n = nx * ny
    k = np.exp(rng.normal(np.log(1e-12), 1.0, n))
    p = I.Problem(dim=2, nx=nx, ny=ny, nz=1, kx=k, ky=k, kz=k, pc_model=pc, pc_pd=5e3, pc_p0=1e4)
    u, uo = I.front_state(p, front_cells=nx / 3.0)
    F, J, (rp, col) = O.assemble(p, u, uo, I.DAY)
    return p, F, J, rp, col


EXACT = dict(coarse_n=10 ** 6)


def _pmat(Mfun, n):
    return np.column_stack([Mfun(e) for e in np.eye(n)])


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_fgmres_reaches_dense_solution(oracle, inputs, kind):
    p, F, J, rp, col = _tiny(inputs, oracle, nx=5, ny=4)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    b = -F
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=kind, amg=oracle.AmgParams(coarse_n=4)))
    x, st, its, rr = oracle.fgmres(rp, col, J, b, M, rtol=1e-12, maxit=200)
    xd = np.linalg.solve(A, b)
    assert st == 0 and rr <= 1e-12
    np.testing.assert_allclose(x, xd, rtol=1e-8, atol=1e-10 * np.abs(xd).max())


def test_unpreconditioned_gmres_converges_within_n(oracle, inputs):
    p, F, J, rp, col = _tiny(inputs, oracle, nx=3, ny=2)
    n = 2 * p.ncell
    x, st, its, rr = oracle.fgmres(rp, col, J, -F, None, m=n, rtol=1e-10, maxit=n + 2)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    assert its <= n
    np.testing.assert_allclose(x, np.linalg.solve(A, -F), rtol=1e-6)


def test_cpr1_equals_m_comb(oracle, inputs):
    """Algorithm 1 == (I - R_p^T A_pp^{-1} R_p (A - P1)) P1^{-1}, no decoupling."""
    p, F, J, rp, col = _tiny(inputs, oracle)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = A.shape[0]
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=1, decouple=0, amg=oracle.AmgParams(**EXACT)))
    got = _pmat(M.apply, n)
    P1 = np.zeros_like(A)
    for i in range(n // 2):
        P1[2 * i:2 * i + 2, 2 * i:2 * i + 2] = A[2 * i:2 * i + 2, 2 * i:2 * i + 2]
    Rp = np.zeros((n // 2, n)); Rp[np.arange(n // 2), 2 * np.arange(n // 2)] = 1
    App = Rp @ A @ Rp.T
    ref = (np.eye(n) - Rp.T @ np.linalg.inv(App) @ Rp @ (A - P1)) @ np.linalg.inv(P1)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


def test_cpr2_equals_m_add(oracle, inputs):
    p, F, J, rp, col = _tiny(inputs, oracle, seed=1)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = A.shape[0]
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=2, decouple=0, amg=oracle.AmgParams(**EXACT)))
    got = _pmat(M.apply, n)
    P1 = np.zeros_like(A)
    for i in range(n // 2):
        P1[2 * i:2 * i + 2, 2 * i:2 * i + 2] = A[2 * i:2 * i + 2, 2 * i:2 * i + 2]
    Rp = np.zeros((n // 2, n)); Rp[np.arange(n // 2), 2 * np.arange(n // 2)] = 1
    Rs = np.zeros((n // 2, n)); Rs[np.arange(n // 2), 2 * np.arange(n // 2) + 1] = 1
    App, Ass = Rp @ A @ Rp.T, Rs @ A @ Rs.T
    C = Rp.T @ np.linalg.inv(App) @ Rp + Rs.T @ np.linalg.inv(Ass) @ Rs
    ref = (np.eye(n) - C @ (A - P1)) @ np.linalg.inv(P1)
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("decouple", [1, 2])
def test_cpr_decoupled_equals_matrix_form_on_scaled_system(oracle, inputs, decouple):
    """With decoupling W (D^{-1} or the quasi-IMPES row combination) the
    preconditioner is M~^{-1} W where M~ is eq. m_comb for W J."""
    p, F, J, rp, col = _tiny(inputs, oracle, seed=2)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = A.shape[0]
    W = np.zeros_like(A)
    for i in range(n // 2):
        blk = A[2 * i:2 * i + 2, 2 * i:2 * i + 2]
        if decouple == 1:
            W[2 * i:2 * i + 2, 2 * i:2 * i + 2] = np.linalg.inv(blk)
        else:
            W[2 * i:2 * i + 2, 2 * i:2 * i + 2] = [[1.0, -blk[0, 1] / blk[1, 1]], [0.0, 1.0]]
    At = W @ A
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=1, decouple=decouple, amg=oracle.AmgParams(**EXACT)))
    got = _pmat(M.apply, n)
    P1 = np.zeros_like(A)
    for i in range(n // 2):
        P1[2 * i:2 * i + 2, 2 * i:2 * i + 2] = At[2 * i:2 * i + 2, 2 * i:2 * i + 2]
    Rp = np.zeros((n // 2, n)); Rp[np.arange(n // 2), 2 * np.arange(n // 2)] = 1
    ref = (np.eye(n) - Rp.T @ np.linalg.inv(Rp @ At @ Rp.T) @ Rp @ (At - P1)) @ np.linalg.inv(P1) @ W
    np.testing.assert_allclose(got, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())


def test_bf_equals_m_bf(oracle, inputs):
    """Algorithm 3 == [[S~^{-1}, -S~^{-1} A_ps A_ss^{-1}], [0, A_ss^{-1}]]."""
    p, F, J, rp, col = _tiny(inputs, oracle, seed=3)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = A.shape[0]
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=3, amg=oracle.AmgParams(**EXACT)))
    got = _pmat(M.apply, n)
    App, Aps, Asp, Ass = A[0::2, 0::2], A[0::2, 1::2], A[1::2, 0::2], A[1::2, 1::2]
    St = App - Aps @ np.diag(1 / np.diag(Ass)) @ Asp
    Si, Ai = np.linalg.inv(St), np.linalg.inv(Ass)
    blk = np.block([[Si, -Si @ Aps @ Ai], [np.zeros_like(Ai), Ai]])
    perm = np.empty(n, dtype=int)
    perm[0::2] = np.arange(n // 2)
    perm[1::2] = n // 2 + np.arange(n // 2)
    ref = blk[np.ix_(perm, perm)]
    np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10 * np.abs(ref).max())


def test_bf_exact_schur_converges_in_two_iterations(oracle, inputs):
    """When A_ss is diagonal the SIMPLE Schur complement is the exact one and,
    with exact inner solves, M is the upper block-triangular factor of Sec. 3.4:
    J M^{-1} = [[I, 0], [A_sp S^{-1}, I]] so (J M^{-1} - I)^2 = 0 and GMRES
    converges in at most two iterations."""
    rng = np.random.default_rng(8)
    p, F, J, rp, col = _tiny(inputs, oracle, nx=5, ny=4, seed=4)
    J = J.copy()
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    off = col != rows
    J[off, 1, 1] = 0.0                      # A_ss diagonal
    J[:, 0, 1] *= 1.0 + 0.3 * rng.standard_normal(J.shape[0])
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = A.shape[0]
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=3, amg=oracle.AmgParams(**EXACT)))
    Minv = _pmat(M.apply, n)
    E = A @ Minv - np.eye(n)
    assert np.abs(E @ E).max() < 1e-8 * max(1.0, np.abs(E).max()) ** 2
    b = inputs.rhs_vector(n, 5)
    x, st, its, rr = oracle.fgmres(rp, col, J, b, M, rtol=1e-10)
    assert st == 0 and its <= 2, its


def test_ilu0_is_exact_on_block_diagonal(oracle, inputs):
    """ILU(0) of a matrix whose pattern admits no fill is its exact LU, so CPR
    with P1 = ILU(0) on a block-diagonal (decoupled cells) J is exact up to the
    pressure correction; here J has no couplings at all, so P1^{-1} = J^{-1}."""
    p, F, J, rp, col = _tiny(inputs, oracle, seed=5)
    rows = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    J = J.copy()
    J[col != rows] = 0.0
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=1, decouple=0, p1=1, amg=oracle.AmgParams(**EXACT)))
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    b = inputs.rhs_vector(A.shape[0], 6)
    np.testing.assert_allclose(M.apply(b), np.linalg.solve(A, b), rtol=1e-10)


def test_newton_converges_quadratically_on_small_grid(oracle, inputs):
    p = inputs.config_small_2d()
    u0 = inputs.initial_state(p)
    u, st, ni, li, hist = oracle.newton(p, u0, u0, inputs.DAY,
                                        oracle.NewtonParams(gmres_rtol=1e-10, prec=oracle.PrecParams(kind=1, decouple=2)))
    assert st == 0, hist
    assert hist[-1] <= 1e-6
    # once in the asymptotic regime the error exponent approaches 2
    h = hist[hist > 1e-9]
    ratios = [np.log(h[k + 1]) / np.log(h[k]) for k in range(len(h) - 1) if h[k] < 1e-2]
    assert any(r > 1.6 for r in ratios), hist
    F, _, _ = oracle.assemble(p, u, u0, inputs.DAY, jacobian=False)
    assert oracle.scaled_fnorm(p, F, inputs.DAY) <= 1e-6


def _lu_parts(oracle, rp, col, lu):
    M = sp.csr_matrix(oracle.bsr2_to_scipy(rp, col, lu))
    L = sp.tril(M, -1, format="csr") + sp.eye(M.shape[0], format="csr")
    U = sp.triu(M, 0, format="csr")
    return L, U


@pytest.mark.parametrize("decouple", [0, 2])
def test_ilu0_factors_match_matrix_on_its_pattern(oracle, inputs, decouple):
    """The defining property of ILU(0) (Saad, Iterative Methods, Sec. 10.3):
    L unit lower and U upper on the pattern of A, with (L U)_ij = a_ij for
    every (i, j) in the pattern. On a 2D gravity Jacobian (raw and
    quasi-IMPES decoupled) fill outside the pattern is dropped, so L U
    differs from A there."""
    p = inputs.config_gravity_2d(10, 2)
    u = inputs.uniform_state(p)
    u = inputs.jitter(u, 4, dp=1e4, ds=0.05)
    F, J, (rp, col) = oracle.assemble(p, u, inputs.uniform_state(p), 4 * inputs.DAY)
    if decouple == 2:
        # quasi-IMPES: pressure row += w * oil row, w = -a_ps,ii / a_ss,ii
        d = J[np.flatnonzero(col == np.repeat(np.arange(rp.size - 1), np.diff(rp)))]
        w = -d[:, 0, 1] / d[:, 1, 1]
        Jt = J.copy()
        Jt[:, 0, :] += np.repeat(w, np.diff(rp))[:, None] * J[:, 1, :]
        J = Jt
    A = sp.csr_matrix(oracle.bsr2_to_scipy(rp, col, J))
    lu = oracle.ilu0(rp, col, J)
    L, U = _lu_parts(oracle, rp, col, lu)
    P = (abs(sp.csr_matrix(oracle.bsr2_to_scipy(rp, col, np.ones_like(J)))) > 0).toarray()
    LU = (L @ U).toarray()
    Ad = A.toarray()
    scale = np.abs(Ad).max(axis=1, keepdims=True)
    assert np.abs((LU - Ad) * P / scale).max() < 1e-12
    assert np.abs((LU - Ad) * ~P / scale).max() > 1e-6      # dropped fill
    b = inputs.rhs_vector(A.shape[0], 8)
    x = oracle.ilu0_solve(rp, col, lu, b)
    xe = sp.linalg.spsolve_triangular(U, sp.linalg.spsolve_triangular(L, b, lower=True), lower=False)
    np.testing.assert_allclose(x, xe, rtol=1e-10, atol=1e-12 * np.abs(xe).max())


def test_ilu0_is_exact_lu_on_a_strip(oracle, inputs):
    """A one-row strip has a block-tridiagonal Jacobian: its LU makes no fill
    outside the pattern, so ILU(0) is the exact LU and the solve is A^{-1}."""
    p = inputs.homogeneous(40, 1).with_(pc_model=2, pc_pd=5e3)
    u, uo = inputs.front_state(p)
    F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    lu = oracle.ilu0(rp, col, J)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    b = inputs.rhs_vector(A.shape[0], 9)
    np.testing.assert_allclose(oracle.ilu0_solve(rp, col, lu, b), np.linalg.solve(A, b), rtol=1e-9,
                               atol=1e-12 * np.abs(np.linalg.solve(A, b)).max())

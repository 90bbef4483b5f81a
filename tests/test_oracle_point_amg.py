"""Pins of the oracle's systems ("point") AMG: black-box AMG on the Jacobian
ordered by grid points (Sec. 3.2), two interleaved unknowns per point.

The pins are a strided-slice definition of the function parts, structural
properties of the hierarchy (shared C/F splitting per point, no
interpolation across functions, Galerkin product), the textbook special
case of a system without cross coupling (it must reduce to scalar AMG on
each function), brute-force checks of the point colouring, and behaviour on
the two-phase Jacobian (hierarchy inside the FP32 range; FGMRES converges).
"""
import numpy as np
import pytest
import scipy.sparse as sp


def _interleave(A0, A1, C01=None, C10=None):
    """Point-ordered matrix with A0 on function 0, A1 on function 1 and
    optional cross couplings C01 (rows of 0, columns of 1) and C10."""
    n = A0.shape[0]
    perm0 = 2 * np.arange(n)
    perm1 = perm0 + 1
    E0 = sp.csr_matrix((np.ones(n), (perm0, np.arange(n))), shape=(2 * n, n))
    E1 = sp.csr_matrix((np.ones(n), (perm1, np.arange(n))), shape=(2 * n, n))
    M = E0 @ A0 @ E0.T + E1 @ A1 @ E1.T
    if C01 is not None:
        M = M + E0 @ C01 @ E1.T
    if C10 is not None:
        M = M + E1 @ C10 @ E0.T
    M = sp.csr_matrix(M)
    M.sort_indices()
    return M


def _poisson(inputs, n):
    rp, c, v = inputs.poisson_2d(n)
    return sp.csr_matrix((v, c, rp), shape=(n * n, n * n))


def test_func_part_is_the_strided_submatrix(oracle):
    rng = np.random.default_rng(3)
    A = sp.random(60, 60, density=0.15, random_state=rng, format="csr") + sp.eye(60)
    A = sp.csr_matrix(A)
    A.sort_indices()
    Ao = oracle.Csr.from_scipy(A)
    for f in (0, 1):
        B = oracle.func_part(Ao, 2, f).scipy().toarray()
        np.testing.assert_array_equal(B, A.toarray()[f::2, f::2])


def _two_phase(oracle, inputs, pc, n):
    p = inputs.config_lognormal_2d(pc, n=n)
    u, uo = inputs.front_state(p)
    F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    A = sp.csr_matrix(oracle.bsr2_to_scipy(rp, col, J))
    A.sort_indices()
    return A, F, J, rp, col


def test_point_hierarchy_structure(oracle, inputs):
    """Shared C/F marks per point; P has only same-function entries, the
    identity on C unknowns, and per function equals the interpolation of that
    function's part under the point splitting; A_{l+1} = P^T A_l P."""
    A, *_ = _two_phase(oracle, inputs, 1e4, 24)
    H = oracle.Amg(oracle.Csr.from_scipy(A), oracle.AmgParams(num_functions=2, coarse_n=40))
    assert H.nlevels >= 3
    for l in range(H.nlevels - 1):
        Al = H.A(l).scipy()
        P = H.P(l).scipy().tocoo()
        cf = H.cf(l)
        np.testing.assert_array_equal(cf[0::2], cf[1::2])
        assert np.all(P.row % 2 == P.col % 2)
        cpts = np.flatnonzero(cf[0::2] == 1)
        Pd = H.P(l).scipy().toarray()
        for f in (0, 1):
            rows = 2 * cpts + f
            np.testing.assert_array_equal(Pd[rows][:, 2 * np.arange(cpts.size) + f], np.eye(cpts.size))
            Af = oracle.func_part(H.A(l), 2, f)
            st = oracle.strength(Af, 0.25)
            Pf = oracle.interp_ext(Af, st, cf[0::2]).scipy().toarray()
            np.testing.assert_array_equal(Pd[f::2, f::2], Pf)
        Ac = (sp.csr_matrix(P).T @ Al @ sp.csr_matrix(P)).toarray()
        np.testing.assert_allclose(H.A(l + 1).scipy().toarray(), Ac, rtol=1e-12,
                                   atol=1e-14 * np.abs(Ac).max())


def test_point_amg_without_cross_coupling_is_scalar_amg_per_function(oracle, inputs):
    """Function 0 = 2D Poisson L, function 1 = 3 L, no coupling between them:
    the point hierarchy coarsens both like scalar AMG on L, and one point
    V-cycle equals scalar V-cycles on L and on 3 L (chunks of 256 points,
    32 on the coarse levels, against scalar chunks of as many rows)."""
    L = _poisson(inputs, 40)
    A = _interleave(L, 3.0 * L)
    Hp = oracle.Amg(oracle.Csr.from_scipy(A), oracle.AmgParams(num_functions=2, chunk=512, chunk_coarse=64))
    H0 = oracle.Amg(oracle.Csr.from_scipy(L), oracle.AmgParams(chunk=256, chunk_coarse=32))
    H1 = oracle.Amg(oracle.Csr.from_scipy(sp.csr_matrix(3.0 * L)), oracle.AmgParams(chunk=256, chunk_coarse=32))
    assert Hp.sizes() == [2 * s for s in H0.sizes()]
    for l in range(H0.nlevels - 1):
        np.testing.assert_array_equal(Hp.cf(l)[0::2], H0.cf(l))
        np.testing.assert_array_equal(Hp.colours(l)[0][0::2], H0.colours(l)[0])
    rng = np.random.default_rng(5)
    b0, b1 = rng.standard_normal(L.shape[0]), rng.standard_normal(L.shape[0])
    b = np.empty(2 * L.shape[0])
    b[0::2], b[1::2] = b0, b1
    x = Hp.vcycle(b)
    np.testing.assert_allclose(x[0::2], H0.vcycle(b0), rtol=1e-11, atol=1e-12 * np.abs(x).max())
    np.testing.assert_allclose(x[1::2], H1.vcycle(b1), rtol=1e-11, atol=1e-12 * np.abs(x).max())


def test_point_colouring_valid_and_first_fit(oracle, inputs):
    """Every unknown of a point has the point's colour; inside a chunk no two
    coupled points share a colour, and each point takes the lowest colour not
    used by coupled earlier points of its chunk."""
    A, *_ = _two_phase(oracle, inputs, 1e3, 30)
    col, nc = oracle.chunk_colour_pt(oracle.Csr.from_scipy(A), 512, 2)
    np.testing.assert_array_equal(col[0::2], col[1::2])
    pc = col[0::2]
    N = A.shape[0] // 2
    Ac = A.tocoo()
    G = sp.csr_matrix((np.ones(Ac.nnz), (Ac.row // 2, Ac.col // 2)), shape=(N, N))
    G = ((G + G.T) != 0).tocsr()
    Crows = 512
    P = Crows // 2
    for p0 in range(0, N, P):
        p1 = min(p0 + P, N)
        for i in range(p0, p1):
            nb = G.indices[G.indptr[i]:G.indptr[i + 1]]
            nb = nb[(nb >= p0) & (nb < p1) & (nb != i)]
            assert not np.any(pc[nb] == pc[i])
            assert set(range(pc[i])) <= set(pc[nb[nb < i]])
    assert nc == pc.max() + 1


def test_point_smoother_sweep_equations(oracle, inputs):
    """After one point-block sweep from zero, every point of the last colour
    of its chunk satisfies its own two equations with the sweep's values
    inside the chunk and the start values (zero) outside."""
    A, *_ = _two_phase(oracle, inputs, 1e4, 20)
    H = oracle.Amg(oracle.Csr.from_scipy(A), oracle.AmgParams(num_functions=2, coarse_n=40))
    assert H.nlevels >= 2
    rng = np.random.default_rng(9)
    b = rng.standard_normal(A.shape[0])
    x = H.smooth(0, b, np.zeros_like(b))
    col, nc = H.colours(0)
    n = A.shape[0]
    Cr = 512
    checked = 0
    for c0 in range(0, n, Cr):
        c1 = min(c0 + Cr, n)
        last = col[c0:c1].max()
        xin = np.zeros(n)
        xin[c0:c1] = x[c0:c1]
        r = b - A @ xin
        for i in range(c0 // 2, c1 // 2):
            if col[2 * i] == last:
                np.testing.assert_allclose(r[2 * i:2 * i + 2], 0.0, atol=1e-9 * np.abs(b).max())
                checked += 1
    assert checked > 0
    assert np.abs(b - A @ x).max() > 1e-3 * np.abs(b).max()


def test_point_hierarchy_inside_fp32_range_where_scalar_overflows(oracle, inputs):
    """On the 256^2 two-phase Jacobian the unknown-agnostic scalar hierarchy
    reaches values beyond the FP32 range (interpolation across the pressure
    and saturation unknowns); the point hierarchy stays far inside it."""
    A, F, J, rp, col = _two_phase(oracle, inputs, 0.0, 256)
    Ms = oracle.Precond(rp, col, J, oracle.PrecParams(kind=oracle.AMG_J_SCALAR, decouple=0))
    Mp = oracle.Precond(rp, col, J, oracle.PrecParams(kind=oracle.AMG_J, decouple=0))
    Hs, Hp = Ms.amg(0), Mp.amg(0)
    mx_s = max(np.abs(Hs.A(l).scipy().data).max() for l in range(Hs.nlevels))
    mx_p = max(np.abs(Hp.A(l).scipy().data).max() for l in range(Hp.nlevels))
    assert mx_s > np.finfo(np.float32).max
    assert mx_p < 1e12


@pytest.mark.parametrize("pc", [0.0, 1e3, 1e4, 1e5])
def test_point_amg_preconditioned_fgmres_converges(oracle, inputs, pc):
    A, F, J, rp, col = _two_phase(oracle, inputs, pc, 64)
    M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=oracle.AMG_J, decouple=0))
    x, st, its, rr = oracle.fgmres(rp, col, J, -F, M, maxit=200)
    assert st == 0 and its <= 60
    assert np.linalg.norm(-F - A @ x) <= 1.0001e-8 * np.linalg.norm(F)

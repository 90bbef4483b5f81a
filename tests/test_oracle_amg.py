"""Pins of the oracle's AMG (Sec. 3.2 with the solver settings of Sec. 4).

Closed forms (1D two-grid), defining properties (strength threshold, PMIS
invariants, valid greedy colouring, Gauss-Seidel equations), library
cross-checks (sparse products against scipy) and convergence behaviour.
"""
import numpy as np
import pytest
import scipy.sparse as sp


def _csr(O, rp, c, v):
    return O.Csr.from_arrays(rp, c, v)


def test_splitmix64_reference_values(oracle):
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: first outputs of the
    # generator as published with the reference Java/C code.
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 2) == 0x06C45D188009454F


def test_strength_hand_example(oracle):
    # row 0: [4, -1, -0.2, -0.5, +0.3]; theta 0.25 -> max 1, threshold 0.25
    # row 1: negative diagonal flips the test: [-1 (col0), -3 (diag), 2 (col2)]
    rows = [[(0, 4.0), (1, -1.0), (2, -0.2), (3, -0.5), (4, 0.3)],
            [(0, -1.0), (1, -3.0), (2, 2.0)],
            [(2, 1.0), (3, 0.5)],
            [(3, 1.0)],
            [(4, 1.0)]]
    rp, c, v = [0], [], []
    for r in rows:
        for j, a in r:
            c.append(j)
            v.append(a)
        rp.append(len(c))
    A = _csr(oracle, rp, c, v)
    s = oracle.strength(A, 0.25)
    expect = [0, 1, 0, 1, 0,      # row 0: -1 and -0.5 strong, -0.2 and +0.3 not
              0, 0, 1,            # row 1 (diag < 0): only +2 is strong
              0, 0,               # row 2: positive off-diagonal, nothing strong
              0, 0]
    assert list(s) == expect


def _random_graph_matrix(n, deg, seed, symmetric):
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=deg / n, random_state=rng, format="csr")
    A.data[:] = -rng.uniform(0.1, 1.0, A.nnz)
    if symmetric:
        A = (A + A.T) * 0.5
    A = A - sp.diags(A.diagonal())
    d = -np.asarray(A.sum(axis=1)).ravel() + 0.1
    A = (A + sp.diags(d)).tocsr()
    A.sort_indices()
    return A


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pmis_symmetric_gives_maximal_independent_set(oracle, seed):
    """With a symmetric strength graph PMIS yields a maximal independent set:
    no two C points are strongly connected and every point that influences
    someone is C or has a strong C neighbour."""
    A = _random_graph_matrix(300, 6, seed, symmetric=True)
    Ao = oracle.Csr.from_scipy(A)
    s = oracle.strength(Ao, 0.0)     # theta 0: every negative coupling is strong
    rp, c, _ = Ao.arrays()
    S = sp.csr_matrix((s.astype(float), c, rp), shape=A.shape)
    S.eliminate_zeros()
    assert (S != S.T).nnz == 0
    cf = oracle.pmis(Ao, s, seed=77, level=0)
    C = cf == 1
    F = cf == -1
    assert np.all(C | F)
    Sb = S.astype(bool)
    assert not (Sb[C][:, C]).nnz
    lam = np.asarray(Sb.sum(axis=0)).ravel()
    has_c = np.asarray(Sb[:, C].sum(axis=1)).ravel() > 0
    assert np.all(has_c[F & (lam > 0)])
    assert np.all(F[lam == 0])


@pytest.mark.parametrize("seed", [4, 5])
def test_pmis_nonsymmetric_invariants(oracle, seed):
    """Every F point that someone depends on strongly depends on a C point;
    points nobody depends on are F; the point with the largest measure is C."""
    A = _random_graph_matrix(400, 5, seed, symmetric=False)
    Ao = oracle.Csr.from_scipy(A)
    s = oracle.strength(Ao, 0.25)
    rp, c, _ = Ao.arrays()
    S = sp.csr_matrix((s.astype(float), c, rp), shape=A.shape).astype(bool)
    cf = oracle.pmis(Ao, s, seed=11, level=3)
    C = cf == 1
    lam = np.asarray(S.sum(axis=0)).ravel()
    dep_on_c = np.asarray(S[:, C].sum(axis=1)).ravel() > 0
    assert np.all(dep_on_c[(cf == -1) & (lam > 0)])
    assert np.all(cf[lam == 0] == -1)
    # largest key wins round one
    keys = [(int(lam[i]) << 24) | (oracle.splitmix64(11, ((2 * 3) << 32) + i) >> 40) for i in range(A.shape[0])]
    top = max(range(A.shape[0]), key=lambda i: (keys[i], -i))
    assert cf[top] == 1


def test_pmis_no_edges_all_fine(oracle):
    A = oracle.Csr.from_scipy(sp.identity(10, format="csr"))
    s = oracle.strength(A, 0.25)
    assert np.all(oracle.pmis(A, s, seed=1) == -1)


def test_two_grid_1d_poisson_closed_form(oracle, inputs):
    """1D Poisson, C points at odd indices: classical interpolation is linear
    interpolation (weights 1/2) and P^T A P = (1/2) tridiag(-1, 2, -1)."""
    n = 15
    rp, c, v = inputs.poisson_1d(n)
    A = _csr(oracle, rp, c, v)
    s = oracle.strength(A, 0.25)
    cf = np.array([1 if i % 2 == 1 else -1 for i in range(n)], dtype=np.int8)
    for P in (oracle.interp(A, s, cf), oracle.interp_ext(A, s, cf)):
        Pd = P.scipy().toarray()
        nc = Pd.shape[1]
        E = np.zeros((n, nc))
        for k in range(nc):
            E[2 * k + 1, k] = 1.0
            E[2 * k, k] = 0.5
            E[2 * k + 2, k] = 0.5
        np.testing.assert_array_equal(Pd, E)
        Ac = oracle.galerkin(A, P).scipy().toarray()
        T = 0.5 * (2 * np.eye(nc) - np.eye(nc, k=1) - np.eye(nc, k=-1))
        np.testing.assert_array_equal(Ac, T)


def test_interpolation_preserves_constants_zero_rowsum(oracle, inputs):
    """For a zero-row-sum M-matrix (Neumann Laplacian) with every connection
    strong, interpolation reproduces constants: P 1 = 1 on interpolated rows."""
    n = 12
    rp, c, v = inputs.poisson_2d(n)
    A = sp.csr_matrix((v, c, rp)).tolil()
    for i in range(n * n):
        A[i, i] = 0.0
        A[i, i] = -A[i].sum()
    A = A.tocsr()
    A.sort_indices()
    Ao = oracle.Csr.from_scipy(A)
    s = oracle.strength(Ao, 0.0)
    cf = oracle.pmis(Ao, s, seed=5)
    for P in (oracle.interp(Ao, s, cf), oracle.interp_ext(Ao, s, cf)):
        Ps = P.scipy()
        rows = np.asarray((Ps != 0).sum(axis=1)).ravel() > 0
        np.testing.assert_allclose((Ps @ np.ones(Ps.shape[1]))[rows], 1.0, rtol=1e-12)


def test_spgemm_and_transpose_match_scipy(oracle):
    rng = np.random.default_rng(3)
    A = sp.random(60, 45, density=0.1, random_state=rng, format="csr")
    B = sp.random(45, 70, density=0.1, random_state=rng, format="csr")
    A.sort_indices(); B.sort_indices()
    C = oracle.spgemm(oracle.Csr.from_scipy(A), oracle.Csr.from_scipy(B)).scipy()
    np.testing.assert_allclose(C.toarray(), (A @ B).toarray(), rtol=1e-14, atol=1e-15)
    T = oracle.transpose(oracle.Csr.from_scipy(A)).scipy()
    np.testing.assert_array_equal(T.toarray(), A.T.toarray())


def _fl(x):
    """Round an exact rational to the nearest double (ties to even)."""
    return float(x)


def test_spgemm_rounding_is_rounded_first_term_then_fused(oracle):
    """Reading R31 of the sparse products: in ascending inner index, the
    first term is the rounded product and every later term is fused into the
    sum (one rounding per term). Checked against exact rational arithmetic on
    terms chosen so that the fused and the separately rounded sums differ in
    the last place, for the product and for the SIMPLE Schur complement."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(11)
    # a 1 x 3 times 3 x 1 product: c = a0 b0 + a1 b1 + a2 b2
    found = 0
    for _ in range(2000):
        a = 1.0 + rng.random(3)
        b = 1.0 + rng.random(3)
        b[1] = -b[1]
        acc = _fl(Fr(a[0]) * Fr(b[0]))
        for k in (1, 2):
            acc = _fl(Fr(a[k]) * Fr(b[k]) + Fr(acc))
        sep = a[0] * b[0]
        for k in (1, 2):
            sep = sep + a[k] * b[k]
        if acc == sep:
            continue
        found += 1
        A = oracle.Csr.from_arrays(np.array([0, 3], np.int32), np.array([0, 1, 2], np.int32), a)
        B = oracle.Csr.from_arrays(np.array([0, 1, 2, 3], np.int32), np.zeros(3, np.int32), b)
        C = oracle.spgemm(A, B).scipy().toarray()
        assert C[0, 0] == acc, (a, b, C[0, 0], acc, sep)
        if found >= 20:
            break
    assert found >= 20
    # S~ = A_pp - A_ps diag(A_ss)^-1 A_sp on 2 x 2 blocks: row 0 of the
    # product is t0 a_sp(0,0) + t1 a_sp(1,0) with t_k = a_ps(0,k) / d_k
    found = 0
    for _ in range(2000):
        aps = 1.0 + rng.random(2)
        asp = 1.0 + rng.random(2)
        asp[1] = -asp[1]
        d = 1.0 + rng.random(2)
        app = 3.0 + rng.random()
        t = aps / d
        acc = _fl(Fr(t[0]) * Fr(asp[0]))
        acc = _fl(Fr(t[1]) * Fr(asp[1]) + Fr(acc))
        sep = t[0] * asp[0] + t[1] * asp[1]
        if acc == sep:
            continue
        found += 1
        I2 = np.array([0, 1, 2], np.int32)
        App = oracle.Csr.from_arrays(I2, np.array([0, 1], np.int32), np.array([app, app]))
        Aps = oracle.Csr.from_arrays(np.array([0, 2, 2], np.int32), np.array([0, 1], np.int32), aps)
        Asp = oracle.Csr.from_arrays(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), asp)
        Ass = oracle.Csr.from_arrays(I2, np.array([0, 1], np.int32), d)
        S = oracle.simple_schur(App, Aps, Asp, Ass).scipy().toarray()
        assert S[0, 0] == app - acc, (S[0, 0], app - acc, app - sep)
        if found >= 20:
            break
    assert found >= 20


def test_galerkin_matches_dense_triple_product(oracle, inputs):
    rp, c, v = inputs.poisson_2d(10)
    A = _csr(oracle, rp, c, v)
    s = oracle.strength(A, 0.25)
    cf = oracle.pmis(A, s, seed=9)
    P = oracle.interp_ext(A, s, cf)
    Pd = P.scipy().toarray()
    Ad = sp.csr_matrix((v, c, rp)).toarray()
    np.testing.assert_allclose(oracle.galerkin(A, P).scipy().toarray(), Pd.T @ Ad @ Pd, rtol=1e-13, atol=1e-13)


def test_simple_schur_matches_dense_formula(oracle, inputs):
    """S~ = A_pp - A_ps diag(A_ss)^{-1} A_sp (eq. SIMPLE-Schur with A_sp)."""
    p = inputs.config_small_2d().with_(nx=8, ny=6, kx=np.full(48, 1e-12), ky=np.full(48, 1e-12), kz=np.full(48, 1e-12))
    u, uo = inputs.front_state(p)
    F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    parts = [oracle.bsr2_part(rp, col, J, r, cc) for r, cc in ((0, 0), (0, 1), (1, 0), (1, 1))]
    S = oracle.simple_schur(*parts).scipy().toarray()
    D = oracle.bsr2_to_scipy(rp, col, J).toarray()
    App, Aps, Asp, Ass = D[0::2, 0::2], D[0::2, 1::2], D[1::2, 0::2], D[1::2, 1::2]
    ref = App - Aps @ np.diag(1.0 / np.diag(Ass)) @ Asp
    np.testing.assert_allclose(S, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


def test_jp_colouring_is_valid_and_greedy(oracle, inputs):
    rp, c, v = inputs.poisson_2d(20)
    A = _csr(oracle, rp, c, v)
    col, nc = oracle.jp_colour(A, seed=3, level=0)
    As = sp.csr_matrix((v, c, rp))
    r, cc = As.nonzero()
    off = r != cc
    assert np.all(col[r[off]] != col[cc[off]])
    assert col.max() + 1 == nc
    # greedy: each lower colour appears among the neighbours
    for i in range(As.shape[0]):
        nb = set(col[As.indices[As.indptr[i]:As.indptr[i + 1]]]) - {col[i]}
        assert set(range(col[i])) <= nb


def test_gauss_seidel_sweep_satisfies_last_colour_rows(oracle, inputs):
    """After a multicolour GS sweep, every row of the last colour holds exactly
    (its unknown was solved last, with all neighbours final)."""
    rp, c, v = inputs.poisson_2d(16)
    A = _csr(oracle, rp, c, v)
    H = oracle.Amg(A, oracle.AmgParams(coarse_n=16))
    col, nc = H.colours(0)
    b = inputs.rhs_vector(256, 2)
    x = H.smooth(0, b, np.zeros(256))
    r = b - sp.csr_matrix((v, c, rp)) @ x
    last = col == nc - 1
    assert np.abs(r[last]).max() < 1e-12
    assert np.abs(r[~last]).max() > 1e-3


def test_vcycle_exact_when_single_level(oracle, inputs):
    rp, c, v = inputs.poisson_2d(9)
    A = _csr(oracle, rp, c, v)
    H = oracle.Amg(A, oracle.AmgParams(coarse_n=1000))
    assert H.nlevels == 1
    b = inputs.rhs_vector(81, 3)
    x = H.vcycle(b)
    np.testing.assert_allclose(sp.csr_matrix((v, c, rp)) @ x, b, rtol=1e-12, atol=1e-12)


def test_dense_lu_against_numpy(oracle):
    rng = np.random.default_rng(0)
    M = rng.standard_normal((30, 30)) + 5 * np.eye(30)
    b = rng.standard_normal(30)
    np.testing.assert_allclose(oracle.dense_lu_solve(M, b), np.linalg.solve(M, b), rtol=1e-12)


def _vcycle_rate(oracle, A, theta, seed=1, smoother=0):
    Ao = oracle.Csr.from_scipy(A)
    H = oracle.Amg(Ao, oracle.AmgParams(theta=theta, smoother=smoother))
    rng = np.random.default_rng(seed)
    b = rng.standard_normal(A.shape[0])
    x = np.zeros_like(b)
    r = b.copy()
    hist = []
    for _ in range(8):
        x = x + H.vcycle(r)
        r = b - A @ x
        hist.append(np.linalg.norm(r))
    return (hist[-1] / hist[1]) ** (1 / 6), H


def test_amg_mesh_independent_on_poisson_2d(oracle, inputs):
    rates = []
    for n in (32, 64, 128, 256):
        rp, c, v = inputs.poisson_2d(n)
        rate, H = _vcycle_rate(oracle, sp.csr_matrix((v, c, rp)), 0.25)
        rates.append(rate)
    assert max(rates) < 0.25, rates
    assert rates[-1] - rates[0] < 0.08, rates


def test_amg_mesh_independent_on_poisson_3d(oracle, inputs):
    rates = []
    for n in (12, 24, 40):
        rp, c, v = inputs.poisson_3d(n)
        rate, H = _vcycle_rate(oracle, sp.csr_matrix((v, c, rp)), 0.5)
        rates.append(rate)
    assert max(rates) < 0.3, rates
    assert rates[-1] - rates[0] < 0.1, rates


@pytest.mark.parametrize("dim", [2, 3])
def test_hybrid_smoother_rate_bounded(oracle, inputs, dim):
    """The hybrid smoother (Gauss-Seidel inside chunks, Jacobi between them)
    keeps the V-cycle rate bounded as the number of chunks grows."""
    sizes = (32, 64, 128) if dim == 2 else (12, 24, 40)
    for n in sizes:
        rp, c, v = inputs.poisson_2d(n) if dim == 2 else inputs.poisson_3d(n)
        rate, H = _vcycle_rate(oracle, sp.csr_matrix((v, c, rp)), 0.25 if dim == 2 else 0.5, smoother=2)
        assert rate < 0.3, (n, rate)


def test_amg_pressure_block_gmres_iterations_flat(oracle, inputs):
    """GMRES + one V-cycle on the pressure Poisson block (A_pp of J at
    S_n = 0, no P_c): iteration counts do not grow with the grid."""
    its = []
    for n in (32, 64, 128):
        p = inputs.homogeneous(n, n).with_(pc_model=0, sn_out=0.0)
        u = inputs.initial_state(p, s_init=0.0)
        u[0::2] += np.linspace(1e3, 0, p.ncell)
        F, J, (rp, col) = oracle.assemble(p, u, u, inputs.DAY)
        M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=oracle.CPR1, decouple=0))
        b = inputs.rhs_vector(2 * p.ncell, 4)
        x, st, it, rr = oracle.fgmres(rp, col, J, b, M)
        assert st == 0
        its.append(it)
    assert max(its) - min(its) <= 3, its


@pytest.mark.parametrize("which", ["poisson2d", "poisson3d", "random"])
def test_chunk_colouring_valid_and_first_fit(oracle, inputs, which):
    """Hybrid-smoother colouring: inside every chunk no two coupled rows share
    a colour, and every row takes the lowest colour not used by the coupled,
    earlier rows of its chunk (first fit); chunks hold `chunk` rows."""
    if which == "poisson2d":
        rp, c, v = inputs.poisson_2d(37)
        A = sp.csr_matrix((v, c, rp))
    elif which == "poisson3d":
        rp, c, v = inputs.poisson_3d(11)
        A = sp.csr_matrix((v, c, rp))
    else:
        A = _random_graph_matrix(1500, 9, 7, symmetric=False)
    col, nc, C = oracle.chunk_colour(oracle.Csr.from_scipy(A), 512)
    assert C == 512   # the chunk parameter itself, whatever the row lengths
    S = ((A + A.T) != 0).tocsr()
    n = A.shape[0]
    for c0 in range(0, n, C):
        c1 = min(c0 + C, n)
        for i in range(c0, c1):
            nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
            nb = nb[(nb >= c0) & (nb < c1) & (nb != i)]
            assert not np.any(col[nb] == col[i])
            earlier = set(col[nb[nb < i]])
            assert set(range(col[i])) <= earlier
    assert nc == col.max() + 1


def test_coarse_levels_use_the_coarse_chunk(oracle, inputs):
    """With chunk_coarse set, level 0 keeps `chunk` and every coarser level
    is coloured and swept in chunks of chunk_coarse rows: its colouring is
    valid and first fit within those chunks, and after one sweep from zero
    the last-colour rows of each chunk satisfy their equations with the
    sweep's values inside the chunk and zero outside."""
    rp, c, v = inputs.poisson_2d(48)
    A0 = sp.csr_matrix((v, c, rp))
    H = oracle.Amg(oracle.Csr.from_scipy(A0), oracle.AmgParams(chunk=512, chunk_coarse=32, coarse_n=20))
    Href = oracle.Amg(oracle.Csr.from_scipy(A0), oracle.AmgParams(chunk=512, chunk_coarse=0, coarse_n=20))
    assert H.sizes() == Href.sizes() and H.nlevels >= 3
    np.testing.assert_array_equal(H.colours(0)[0], Href.colours(0)[0])
    for l in range(1, H.nlevels - 1):
        A = H.A(l).scipy().tocsr()
        col, nc = H.colours(l)
        n = A.shape[0]
        S = ((A + A.T) != 0).tocsr()
        for c0 in range(0, n, 32):
            c1 = min(c0 + 32, n)
            for i in range(c0, c1):
                nb = S.indices[S.indptr[i]:S.indptr[i + 1]]
                nb = nb[(nb >= c0) & (nb < c1) & (nb != i)]
                assert not np.any(col[nb] == col[i])
                assert set(range(col[i])) <= set(col[nb[nb < i]])
        rng = np.random.default_rng(l)
        b = rng.standard_normal(n)
        x = H.smooth(l, b, np.zeros(n))
        checked = 0
        for c0 in range(0, n, 32):
            c1 = min(c0 + 32, n)
            last = col[c0:c1].max()
            xin = np.zeros(n)
            xin[c0:c1] = x[c0:c1]
            r = b - A @ xin
            rows = [i for i in range(c0, c1) if col[i] == last]
            np.testing.assert_allclose(r[rows], 0.0, atol=1e-10 * np.abs(b).max())
            checked += len(rows)
        assert checked > 0

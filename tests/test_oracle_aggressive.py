"""Pins of the oracle's aggressive coarsening (two-stage form, the remaining
half of the PMIS follow-up: fewer levels and lower operator complexity).

With agg_levels = k the first k coarse grids are each two coarsening stages:
level l interpolates from level l+2 of the ordinary hierarchy with the
product of the two stages' interpolations, and level l+1 is dropped. Pinned
against the ordinary hierarchy (same splittings and operators, P equal to
the library product of the two stages, C iff C in both stages), and by what
aggressive coarsening is for: operator complexity down from ~2.5 to ~1.5 on
2D Poisson, V-cycle still convergent and mesh-independent, FGMRES still
converging on the two-phase Jacobian in point mode.
"""
import numpy as np
import pytest
import scipy.sparse as sp


def _poisson(inputs, n):
    rp, c, v = inputs.poisson_2d(n)
    return sp.csr_matrix((v, c, rp), shape=(n * n, n * n))


def _rate(H, A, its=15):
    rng = np.random.default_rng(0)
    b = rng.standard_normal(A.shape[0])
    x = np.zeros_like(b)
    rs = []
    for _ in range(its):
        x = x + H.vcycle(b - A @ x)
        rs.append(np.linalg.norm(b - A @ x))
    return (rs[-1] / rs[-6]) ** 0.2


@pytest.mark.parametrize("nfun", [1, 2])
def test_aggressive_levels_are_the_ordinary_ones_with_stages_merged(oracle, inputs, nfun):
    if nfun == 1:
        A = _poisson(inputs, 64)
    else:
        p = inputs.config_lognormal_2d(1e4, n=40)
        u, uo = inputs.front_state(p)
        F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
        A = sp.csr_matrix(oracle.bsr2_to_scipy(rp, col, J))
        A.sort_indices()
    Ao = oracle.Csr.from_scipy(A)
    H0 = oracle.Amg(Ao, oracle.AmgParams(num_functions=nfun, coarse_n=40))
    H1 = oracle.Amg(Ao, oracle.AmgParams(num_functions=nfun, coarse_n=40, agg_levels=1))
    H2 = oracle.Amg(Ao, oracle.AmgParams(num_functions=nfun, coarse_n=40, agg_levels=2))
    s0 = H0.sizes()
    assert len(s0) >= 5
    assert H1.sizes() == [s0[0]] + s0[2:]
    assert H2.sizes() == [s0[0], s0[2]] + s0[4:]
    for l in range(2, H0.nlevels):
        np.testing.assert_array_equal(H1.A(l - 1).scipy().toarray(), H0.A(l).scipy().toarray())
    P = H1.P(0).scipy()
    Pref = (H0.P(0).scipy() @ H0.P(1).scipy()).toarray()
    np.testing.assert_allclose(P.toarray(), Pref, rtol=1e-13, atol=1e-15 * np.abs(Pref).max())
    cf0, cf1 = H0.cf(0), H0.cf(1)
    expect = np.full(cf0.size, -1, np.int8)
    expect[cf0 == 1] = cf1
    np.testing.assert_array_equal(H1.cf(0), expect)
    # level 1 onwards of the one-stage-merged hierarchy is the ordinary one from level 2
    np.testing.assert_array_equal(H1.P(1).scipy().toarray(), H0.P(2).scipy().toarray())
    P2 = (H0.P(2).scipy() @ H0.P(3).scipy()).toarray()
    np.testing.assert_allclose(H2.P(1).scipy().toarray(), P2, rtol=1e-13, atol=1e-15 * np.abs(P2).max())
    if nfun == 2:
        Pc = P.tocoo()
        assert np.all(Pc.row % 2 == Pc.col % 2)          # still no interpolation across functions


def test_aggressive_coarsening_complexity_and_convergence(oracle, inputs):
    """2D Poisson: operator complexity ~2.5 -> ~1.5; the V-cycle stays a
    convergent, mesh-independent iteration (factor <= 0.7 at 64^2..256^2)."""
    for n in (64, 128, 256):
        A = _poisson(inputs, n)
        Ao = oracle.Csr.from_scipy(A)
        H0 = oracle.Amg(Ao, oracle.AmgParams())
        H1 = oracle.Amg(Ao, oracle.AmgParams(agg_levels=1))
        c0 = sum(H0.A(l).info()[2] for l in range(H0.nlevels)) / A.nnz
        c1 = sum(H1.A(l).info()[2] for l in range(H1.nlevels)) / A.nnz
        assert c0 > 2.2 and c1 < 1.7, (n, c0, c1)
        assert _rate(H1, A) <= 0.7


def test_aggressive_point_amg_preconditions_fgmres(oracle, inputs):
    p = inputs.config_lognormal_2d(1e3, n=48)
    u, uo = inputs.front_state(p)
    F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    its = {}
    for agg in (0, 1):
        M = oracle.Precond(rp, col, J, oracle.PrecParams(kind=0, decouple=0, amg=oracle.AmgParams(agg_levels=agg)))
        x, st, it, rr = oracle.fgmres(rp, col, J, -F, M, maxit=400)
        assert st == 0
        its[agg] = it
    assert its[1] <= 3 * its[0] + 10, its

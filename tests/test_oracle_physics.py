"""Pins of the oracle's discrete model (Sec. 2) and exact Jacobian (Sec. 3.1).

Each check compares the oracle with something other than itself: hand
values, finite differences of its own residual, conservation identities
and the textbook TPFA Laplacian.
"""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _small(I, dim=2, nx=6, ny=5, nz=1, pc_model=2, g=0.0, seed=0):
    rng = np.random.default_rng(1234 + seed)
    n = nx * ny * nz
    k = np.exp(rng.normal(np.log(1e-12), 1.0, n))
    p = I.Problem(dim=dim, nx=nx, ny=ny, nz=nz, kx=k, ky=k * 0.7, kz=k * 0.1,
                  pc_model=pc_model, pc_pd=5e3, pc_p0=2e4, bc_lambda=2.0, g=g)
    u, uo = I.front_state(p, front_cells=nx / 3.0)
    u = I.jitter(u, seed)
    uo = I.jitter(uo, seed + 100)
    u[1::2] = np.clip(u[1::2], 0.12, 0.88)
    uo[1::2] = np.clip(uo[1::2], 0.12, 0.88)
    return p, u, uo


def test_constitutive_hand_values(oracle, inputs):
    with open(os.path.join(GOLD, "constitutive.json")) as f:
        gold = json.load(f)
    for c in gold["cases"]:
        p = inputs.homogeneous(2, 2).with_(bc_lambda=c["bc_lambda"], mu_w=c["mu_w"], mu_n=c["mu_n"],
                                           pc_model=c["pc_model"], pc_pd=c["pc_pd"], pc_p0=c["pc_p0"])
        o = oracle.constitutive(p, c["sn"])
        np.testing.assert_allclose(o[0], c["lambda_w"], rtol=1e-13)
        np.testing.assert_allclose(o[1], c["lambda_n"], rtol=1e-13)
        np.testing.assert_allclose(o[4], c["pc"], rtol=1e-13, atol=1e-12)


def test_two_cell_fluxes_hand_values(oracle, two_cell_cases):
    """Sec. 2 on two cells with K_0 != K_1: the face permeability is the
    harmonic average and each phase's mobility comes from the cell its flow
    leaves (the other cell at a tie), checked against hand-derived fluxes
    in both flow directions, with the phases flowing opposite ways, and
    along z in 3D. An arithmetic face average or a flipped upwind test
    misses these values by 25 % or more."""
    cases, dt = two_cell_cases
    for c, p, u in cases:
        F, J, (rp, col) = oracle.assemble(p, u, u, dt)
        np.testing.assert_allclose(F[:2], c["F0"], rtol=1e-12, atol=1e-20, err_msg=c["name"])
        if "J00_pw_pw" in c:
            assert list(col[rp[0]:rp[1]]) == [0, 1]
            np.testing.assert_allclose(J[rp[0], 0, 0], c["J00_pw_pw"], rtol=1e-12, err_msg=c["name"])
            np.testing.assert_allclose(J[rp[0] + 1, 0, 0], c["J01_pw_pw"], rtol=1e-12, err_msg=c["name"])


@pytest.mark.parametrize("pc_model", [0, 1, 2])
def test_constitutive_derivatives_fd(oracle, inputs, pc_model):
    p = inputs.homogeneous(2, 2).with_(pc_model=pc_model, pc_pd=5e3, pc_p0=2e4, bc_lambda=2.5)
    for sn in [0.05, 0.3, 0.61, 0.93]:
        h = 1e-7
        d = (oracle.constitutive(p, sn + h) - oracle.constitutive(p, sn - h)) / (2 * h)
        o = oracle.constitutive(p, sn)
        np.testing.assert_allclose(o[2], d[0], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(o[3], d[1], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(o[5], d[4], rtol=1e-6, atol=1e-6)


def test_brooks_corey_linear_continuation(oracle, inputs):
    """Below Sb = 1e-4 P_c continues linearly with the slope at 1e-4."""
    p = inputs.homogeneous(2, 2).with_(pc_model=2, pc_pd=5e3, bc_lambda=2.0)
    eps = 1e-4
    pe = 5e3 * eps ** -0.5
    slope_sb = -(5e3 / 2.0) * eps ** -1.5          # dPc/dSb at eps
    for sb in [5e-5, 1e-6, 0.0]:
        o = oracle.constitutive(p, 1.0 - sb)
        np.testing.assert_allclose(o[4], pe + slope_sb * (sb - eps), rtol=1e-12)
        np.testing.assert_allclose(o[5], -slope_sb, rtol=1e-12)


@pytest.mark.parametrize("case", [
    dict(dim=2, nx=6, ny=5, nz=1, pc_model=2, g=0.0),
    dict(dim=2, nx=5, ny=4, nz=1, pc_model=1, g=9.81),
    dict(dim=2, nx=4, ny=4, nz=1, pc_model=0, g=0.0),
    dict(dim=3, nx=4, ny=3, nz=3, pc_model=2, g=9.81),
])
def test_jacobian_matches_finite_differences(oracle, inputs, case):
    """Exact J (eq. linearize_fc) against central differences of F."""
    p, u, uo = _small(inputs, **case)
    F0, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = u.size
    Jfd = np.zeros((n, n))
    for k in range(n):
        h = 1e-3 if k % 2 == 0 else 1e-8
        up, um = u.copy(), u.copy()
        up[k] += h
        um[k] -= h
        Fp = oracle.assemble(p, up, uo, inputs.DAY, pattern=(rp, col), jacobian=False)[0]
        Fm = oracle.assemble(p, um, uo, inputs.DAY, pattern=(rp, col), jacobian=False)[0]
        Jfd[:, k] = (Fp - Fm) / (2 * h)
    scale = np.abs(A).max(axis=0, keepdims=True)
    err = np.abs(A - Jfd) / scale
    assert err.max() < 1e-6, err.max()
    # sparsity: nothing outside the TPFA block pattern
    assert np.all(Jfd[np.abs(A) == 0] == 0) or np.abs(Jfd[np.abs(A) == 0]).max() < 1e-12 * scale.max()


def test_mass_conservation_interior_fluxes_cancel(oracle, inputs):
    """Summed over cells, interior TPFA fluxes cancel: sum F_a = storage - injection
    when the outlet face carries no flux (outlet cells at outlet conditions, g = 0)."""
    p, u, uo = _small(inputs, nx=7, ny=6, pc_model=2)
    p = p.with_(sn_out=0.3)
    out = (np.arange(p.ncell) % p.nx) == p.nx - 1
    u[0::2][out] = p.p_out
    u[1::2][out] = p.sn_out
    F, _, _ = oracle.assemble(p, u, uo, inputs.DAY, jacobian=False)
    V = p.hx * p.hy * 1.0
    stor_w = V * p.phi * p.rho_w * ((1 - u[1::2]) - (1 - uo[1::2])).sum() / inputs.DAY
    stor_n = V * p.phi * p.rho_n * (u[1::2] - uo[1::2]).sum() / inputs.DAY
    inj = p.rho_w * p.u_in * p.hy * 1.0 * p.ny
    flux_scale = np.abs(F).max()
    np.testing.assert_allclose(F[0::2].sum(), stor_w - inj, atol=1e-11 * flux_scale * p.ncell)
    np.testing.assert_allclose(F[1::2].sum(), stor_n, atol=1e-11 * flux_scale * p.ncell)


def test_uniform_state_has_zero_residual(oracle, inputs):
    p = inputs.homogeneous(5, 4).with_(u_in=0.0, pc_model=2, pc_pd=5e3)
    u = inputs.initial_state(p, s_init=p.sn_out)
    F, J, _ = oracle.assemble(p, u, u, inputs.DAY)
    assert np.all(F == 0.0)
    # storage-only residual when only S_old differs
    uo = u.copy()
    uo[1::2] += 0.01
    F, _, _ = oracle.assemble(p, u, uo, inputs.DAY)
    V = 1.0
    np.testing.assert_allclose(F[0::2], V * p.phi * p.rho_w * 0.01 / inputs.DAY, rtol=1e-12)
    np.testing.assert_allclose(F[1::2], -V * p.phi * p.rho_n * 0.01 / inputs.DAY, rtol=1e-12)


def test_single_phase_limit_is_textbook_tpfa_laplacian(oracle, inputs):
    """S_n = 0 (k_rw = 1, k_rn = 0) and no P_c: A_pp is (K rho_w / mu_w) times the
    5-point TPFA Laplacian with the half-cell Dirichlet term on the outlet face."""
    nx, ny, K = 6, 5, 2e-12
    p = inputs.homogeneous(nx, ny, K).with_(pc_model=0, sn_out=0.0)
    u = inputs.initial_state(p, s_init=0.0)
    u[0::2] += np.linspace(1e3, 0, p.ncell)
    F, J, (rp, col) = oracle.assemble(p, u, u, inputs.DAY)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()[0::2, 0::2]
    L = np.zeros((p.ncell, p.ncell))
    for iy in range(ny):
        for ix in range(nx):
            i = ix + nx * iy
            for jx, jy in ((ix - 1, iy), (ix + 1, iy), (ix, iy - 1), (ix, iy + 1)):
                if 0 <= jx < nx and 0 <= jy < ny:
                    L[i, i] += 1.0
                    L[i, jx + nx * jy] -= 1.0
            if ix == nx - 1:
                L[i, i] += 2.0
    np.testing.assert_allclose(A, (K * p.rho_w / p.mu_w) * L, rtol=1e-13, atol=0)


def test_jacobian_block_structure(oracle, inputs):
    """Sec. 3.1 list: A_pp is an M-matrix-like elliptic block (positive
    diagonal, non-positive off-diagonals, weakly diagonally dominant)."""
    p = inputs.config_small_2d()
    u, uo = inputs.front_state(p)
    F, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    App = A[0::2, 0::2]
    d = np.diag(App)
    off = App - np.diag(d)
    assert np.all(d > 0)
    assert np.all(off <= 0)
    assert np.all(d + off.sum(axis=1) >= -1e-12 * d)


def _wells(p):
    """Corner wells of the examples of Sec. 4 on grid p: injection in cell 0
    (top-left: depth grows with iy), outlet on the x = L face of the top-right
    cell."""
    return p.with_(well_in=0, well_out=p.nx - 1, q_in=5.0 / 86400.0)


@pytest.mark.parametrize("case", [
    dict(dim=2, nx=6, ny=5, nz=1, pc_model=2, g=9.81),
    dict(dim=3, nx=4, ny=3, nz=3, pc_model=1, g=9.81),
])
def test_jacobian_with_point_wells_matches_finite_differences(oracle, inputs, case):
    p, u, uo = _small(inputs, **case)
    p = _wells(p)
    F0, J, (rp, col) = oracle.assemble(p, u, uo, inputs.DAY)
    A = oracle.bsr2_to_scipy(rp, col, J).toarray()
    n = u.size
    Jfd = np.zeros((n, n))
    for k in range(n):
        h = 1e-3 if k % 2 == 0 else 1e-8
        up, um = u.copy(), u.copy()
        up[k] += h
        um[k] -= h
        Fp = oracle.assemble(p, up, uo, inputs.DAY, pattern=(rp, col), jacobian=False)[0]
        Fm = oracle.assemble(p, um, uo, inputs.DAY, pattern=(rp, col), jacobian=False)[0]
        Jfd[:, k] = (Fp - Fm) / (2 * h)
    scale = np.abs(A).max(axis=0, keepdims=True)
    assert (np.abs(A - Jfd) / scale).max() < 1e-6


def test_point_wells_mass_balance(oracle, inputs):
    """Summed over cells, with the outlet cell at outlet conditions and g = 0:
    sum F_w = storage - rho_w q_in, sum F_n = storage; and only the well cells
    differ from the face-condition residual apart from the old face cells."""
    p, u, uo = _small(inputs, nx=7, ny=6, pc_model=2)
    p = _wells(p).with_(sn_out=0.3)
    u[2 * p.well_out] = p.p_out
    u[2 * p.well_out + 1] = p.sn_out
    F, _, _ = oracle.assemble(p, u, uo, inputs.DAY, jacobian=False)
    V = p.hx * p.hy * 1.0
    stor_w = V * p.phi * p.rho_w * ((1 - u[1::2]) - (1 - uo[1::2])).sum() / inputs.DAY
    stor_n = V * p.phi * p.rho_n * (u[1::2] - uo[1::2]).sum() / inputs.DAY
    flux_scale = np.abs(F).max()
    np.testing.assert_allclose(F[0::2].sum(), stor_w - p.rho_w * p.q_in, atol=1e-11 * flux_scale * p.ncell)
    np.testing.assert_allclose(F[1::2].sum(), stor_n, atol=1e-11 * flux_scale * p.ncell)
    # the face-condition problem differs from the well problem only in the
    # x = 0 cells (injection) and the x = L cells (outlet)
    Ff, _, _ = oracle.assemble(p.with_(well_in=-1, well_out=-1), u, uo, inputs.DAY, jacobian=False)
    ix = np.arange(p.ncell) % p.nx
    same = (ix != 0) & (ix != p.nx - 1)
    np.testing.assert_array_equal(F[0::2][same], Ff[0::2][same])
    np.testing.assert_array_equal(F[1::2][same], Ff[1::2][same])

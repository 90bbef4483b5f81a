"""The seeded synthetic inputs follow the recipes they stand for (the
stand-ins for the paper's SPE10 data): log-normal fields with the stated
sample mean and spread, the layered 3D grid's layers constant in z with
kz = 0.1 kx, the channelised 3D grid's 30 % channels with a 1e4
permeability contrast, reproducible seeds, and windows that cut the same
values out of a larger grid. Small sizes, no GPU."""
import numpy as np
import pytest

from paper_1611_00127_gb300 import inputs as I


def test_lognormal_2d_mean_spread_and_seed():
    p = I.config_lognormal_2d(1e4, n=64)
    lnk = np.log(p.kx)
    assert lnk.mean() == pytest.approx(np.log(1e-12), abs=1e-9)
    assert lnk.std() == pytest.approx(2.0, rel=1e-9)
    assert np.array_equal(p.kx, p.ky) and np.array_equal(p.kx, p.kz)
    assert p.pc_model == I.PC_BROOKS_COREY and p.pc_pd == 1e4
    # seeded: the same call gives the same field, another member another one
    assert np.array_equal(I.config_lognormal_2d(1e4, n=64).kx, p.kx)
    assert not np.array_equal(I.config_lognormal_2d(1e4, n=64, member=1).kx, p.kx)
    assert I.config_lognormal_2d(0.0, n=64).pc_model == I.PC_NONE


def test_lognormal_field_is_correlated_over_ell():
    rng = np.random.default_rng(1)
    f = I.lognormal_field((256, 256), 1.0, 8.0, 0.0, rng)
    # neighbour correlation of a Gaussian-smoothed field with covariance
    # exp(-r^2 / (2 ell^2)) at r = 1, 8: about 0.99 and 0.61
    c1 = np.corrcoef(f[:, :-1].ravel(), f[:, 1:].ravel())[0, 1]
    c8 = np.corrcoef(f[:, :-8].ravel(), f[:, 8:].ravel())[0, 1]
    assert c1 > 0.95
    assert 0.45 < c8 < 0.75


def test_layered_3d_layers_and_anisotropy():
    n, layers = 32, 8
    p = I.config_layered_3d(n=n, layers=layers)
    kx = p.kx.reshape(n, n, n)
    per = n // layers
    for l in range(layers):
        blk = kx[l * per:(l + 1) * per]
        assert np.all(blk == blk[0][None, :, :])          # constant in z within a layer
    assert not np.array_equal(kx[0], kx[per])               # layers differ
    np.testing.assert_allclose(p.kz, 0.1 * p.kx, rtol=1e-15)
    assert np.array_equal(p.ky, p.kx)
    assert np.log(kx[0]).std() == pytest.approx(3.0, rel=1e-9)


def test_channel_3d_fraction_and_contrast():
    n = 32
    p = I.config_channel_3d(n=n)
    k = p.kx
    # the two facies sit 1e4 apart, each scaled by exp(N(0,1)) noise: the
    # channel cells are the 30 % with k above the geometric midpoint 1e-13
    chan = k > 1e-13
    assert chan.mean() == pytest.approx(0.30, abs=0.01)
    ratio = np.exp(np.log(k[chan]).mean() - np.log(k[~chan]).mean())
    assert 3e3 < ratio < 3e4
    assert np.array_equal(I.config_channel_3d(n=n).kx, k)


def test_window_cuts_the_corner_block():
    p = I.config_channel_3d(n=32)
    w = I.window(p, 8, 4, 2)
    assert (w.nx, w.ny, w.nz, w.dim) == (8, 4, 2, 3)
    full = p.kx.reshape(32, 32, 32)
    np.testing.assert_array_equal(w.kx.reshape(2, 4, 8), full[:2, :4, :8])
    assert w.well_in == -1 and w.well_out == -1
    with pytest.raises(ValueError):
        I.window(p, 33, 1, 1)

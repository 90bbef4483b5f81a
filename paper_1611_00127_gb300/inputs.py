"""Seeded synthetic workloads for the two-phase porous-media Jacobian solves.

This module only generates input data: grids, permeability fields, fluid and
rock constants, and the (p_w, S_n) states at which a Jacobian is formed. It
holds none of the solver arithmetic (no residual, no Jacobian, no AMG), so
both the CUDA path and the CPU oracle can take their inputs from it.

The paper's heterogeneous cases use SPE10 permeability (Sec. 4, Sec. 4.1),
which is not available here. Seeded log-normal Gaussian random fields of the
same kind stand in for it; the recipes are:

* ``lognormal_field``: white noise convolved with a Gaussian kernel of
  standard deviation ell/sqrt(2) (so the covariance is exp(-r^2 / 2 ell^2)),
  truncated at 4 kernel standard deviations, periodic wrap, then shifted and
  scaled to the requested sample mean and standard deviation of ln k.
* 2D single-Jacobian grids: 32x32 homogeneous (k = 1e-12 m^2) and 256x256
  log-normal (sigma 2, ell 8 cells, mean ln 1e-12).
* 3D layered 128^3: 8 layers of 16 z-cells, each layer its own 2D field
  (sigma 3, ell 8), constant in z inside the layer, kz = 0.1 kx.
* Ensemble: 96 square 2D grids with sides drawn from {64,...,512}, each with
  its own field and sigma ~ U[1, 3].
* 3D channelised 256^3: a 3D field with ell = (64, 8, 4) cells thresholded at
  its 70th percentile gives 30 % channel cells; k = 1e-11 in channels and
  1e-15 elsewhere, times exp of a unit-variance field with ell = 8.

Fluid constants follow the paper's Table of input data (Sec. 4.1): water
density 1000 and oil density 700 kg/m^3, porosity 0.2; viscosities come
from the workload (1e-3 and 5e-3 Pa s). Cells are 1 m cubes; a 2D grid is one
1 m thick layer. Time step 1 day.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

BASE_SEED = 20161101
DAY = 86400.0

PC_NONE = 0
PC_LINEAR = 1
PC_BROOKS_COREY = 2


@dataclass
class Problem:
    """One Cartesian grid with its permeability and constitutive constants.

    Cells are numbered lexicographically, x fastest: i = ix + nx*(iy + ny*iz).
    Unknowns are interleaved per cell as (p_w [Pa], S_n [-]).
    """

    dim: int
    nx: int
    ny: int
    nz: int
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray
    hx: float = 1.0
    hy: float = 1.0
    hz: float = 1.0
    phi: float = 0.2
    mu_w: float = 1e-3
    mu_n: float = 5e-3
    rho_w: float = 1000.0
    rho_n: float = 700.0
    g: float = 0.0
    pc_model: int = PC_BROOKS_COREY
    pc_p0: float = 0.0
    pc_pd: float = 5e3
    bc_lambda: float = 2.0
    s_wr: float = 0.0
    s_nr: float = 0.0
    u_in: float = 1e-6       # injected water Darcy flux through the x = 0 face [m/s]
    p_out: float = 1e5       # Dirichlet water pressure on the x = L face [Pa]
    sn_out: float = 0.1      # oil saturation of fluid entering through x = L
    q_in: float = 0.0        # point-well water rate into cell `well_in` [m^3/s]
    well_in: int = -1        # injection cell (-1: through the x = 0 face at u_in)
    well_out: int = -1       # outlet cell on x = L (-1: the whole x = L face)
    name: str = ""

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def ndof(self) -> int:
        return 2 * self.ncell

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _rng(*keys: int) -> np.random.Generator:
    return np.random.default_rng([BASE_SEED, *[int(k) for k in keys]])


def lognormal_field(shape: Tuple[int, ...], sigma: float, ell, mean: float,
                    rng: np.random.Generator) -> np.ndarray:
    """Gaussian random field with sample mean ``mean`` and sample std ``sigma``.

    ``shape`` is in array order (z, y, x) or (y, x); ``ell`` is a scalar or a
    per-axis correlation length in cells given in the same order.
    """
    from scipy.ndimage import gaussian_filter

    white = rng.standard_normal(shape)
    ell_arr = np.broadcast_to(np.asarray(ell, dtype=np.float64), (len(shape),))
    smooth = gaussian_filter(white, sigma=tuple(ell_arr / np.sqrt(2.0)),
                             mode="wrap", truncate=4.0)
    smooth = smooth - smooth.mean()
    sd = smooth.std()
    if sd > 0:
        smooth = smooth / sd
    return mean + sigma * smooth


def homogeneous(nx: int, ny: int, k: float = 1e-12, nz: int = 1) -> Problem:
    n = nx * ny * nz
    kk = np.full(n, k, dtype=np.float64)
    return Problem(dim=2 if nz == 1 else 3, nx=nx, ny=ny, nz=nz,
                   kx=kk.copy(), ky=kk.copy(), kz=kk.copy())


def config_small_2d() -> Problem:
    """32x32 homogeneous grid, Brooks-Corey lambda 2, entry pressure 5e3 Pa."""
    p = homogeneous(32, 32, 1e-12)
    return p.with_(pc_model=PC_BROOKS_COREY, pc_pd=5e3, bc_lambda=2.0,
                   name="2d_32x32_homogeneous_bc")


def config_lognormal_2d(pc_scale: float, n: int = 256, sigma: float = 2.0,
                        ell: float = 8.0, member: int = 0) -> Problem:
    """n x n log-normal field; Brooks-Corey entry pressure = pc_scale (0: no Pc)."""
    rng = _rng(2, member)
    lnk = lognormal_field((n, n), sigma, ell, np.log(1e-12), rng)
    k = np.exp(lnk).reshape(-1).astype(np.float64)
    model = PC_NONE if pc_scale == 0 else PC_BROOKS_COREY
    return Problem(dim=2, nx=n, ny=n, nz=1, kx=k, ky=k.copy(), kz=k.copy(),
                   pc_model=model, pc_pd=float(pc_scale), bc_lambda=2.0,
                   name=f"2d_{n}x{n}_lognormal_pc{pc_scale:g}")


PC_SCALES_2D = (0.0, 1e3, 1e4, 1e5)


def config_layered_3d(n: int = 128, layers: int = 8, sigma: float = 3.0,
                      ell: float = 8.0, anis: float = 0.1,
                      pc_scale: float = 5e3) -> Problem:
    """n^3 grid of `layers` log-normal layers, kz = anis * kx."""
    rng = _rng(3)
    per = n // layers
    kx = np.empty((n, n, n), dtype=np.float64)
    for l in range(layers):
        lnk = lognormal_field((n, n), sigma, ell, np.log(1e-12), rng)
        z0 = l * per
        z1 = n if l == layers - 1 else (l + 1) * per
        kx[z0:z1] = np.exp(lnk)[None, :, :]
    kx = kx.reshape(-1)
    return Problem(dim=3, nx=n, ny=n, nz=n, kx=kx, ky=kx.copy(), kz=anis * kx,
                   pc_model=PC_BROOKS_COREY, pc_pd=pc_scale, bc_lambda=2.0,
                   name=f"3d_{n}^3_layered")


ENSEMBLE_SIDES = (64, 96, 128, 192, 256, 384, 512)


def config_ensemble(count: int = 96, sides=ENSEMBLE_SIDES,
                    pc_scale: float = 1e4) -> List[Problem]:
    """`count` independent 2D grids with seeded sides and field strengths."""
    rng = _rng(4)
    chosen = rng.choice(np.asarray(sides), size=count)
    sig = rng.uniform(1.0, 3.0, size=count)
    out = []
    for m in range(count):
        n = int(chosen[m])
        frng = _rng(4, 1000 + m)
        lnk = lognormal_field((n, n), float(sig[m]), 8.0, np.log(1e-12), frng)
        k = np.exp(lnk).reshape(-1)
        out.append(Problem(dim=2, nx=n, ny=n, nz=1, kx=k, ky=k.copy(),
                           kz=k.copy(), pc_model=PC_BROOKS_COREY,
                           pc_pd=pc_scale, bc_lambda=2.0,
                           name=f"ens{m}_{n}x{n}_s{sig[m]:.2f}"))
    return out


def config_channel_3d(n: int = 256, pc_scale: float = 1e4) -> Problem:
    """n^3 binary-facies channel field (30 % channels, k ratio 1e4) with noise."""
    rng = _rng(5)
    shape = (n, n, n)  # (z, y, x)
    facies = lognormal_field(shape, 1.0, (4.0, 8.0, 64.0), 0.0, rng)
    thr = np.percentile(facies, 70.0)
    chan = facies >= thr
    noise = lognormal_field(shape, 1.0, 8.0, 0.0, rng)
    k = np.where(chan, 1e-11, 1e-15) * np.exp(noise)
    k = k.reshape(-1).astype(np.float64)
    return Problem(dim=3, nx=n, ny=n, nz=n, kx=k, ky=k.copy(), kz=k.copy(),
                   pc_model=PC_BROOKS_COREY, pc_pd=pc_scale, bc_lambda=2.0,
                   name=f"3d_{n}^3_channel")


def window(p: Problem, nx: int, ny: int, nz: int) -> Problem:
    """The corner block of cells ix < nx, iy < ny, iz < nz of a grid as a
    grid of its own (same permeability values and constants). Used to time
    the CPU oracle on a bounded part of a field too large for it."""
    if not (1 <= nx <= p.nx and 1 <= ny <= p.ny and 1 <= nz <= p.nz):
        raise ValueError("window larger than the grid")

    def cut(a):
        return np.ascontiguousarray(a.reshape(p.nz, p.ny, p.nx)[:nz, :ny, :nx]).reshape(-1)

    dim = 3 if nz > 1 or p.dim == 3 else 2
    return dataclasses.replace(p, dim=dim, nx=nx, ny=ny, nz=nz, kx=cut(p.kx), ky=cut(p.ky), kz=cut(p.kz),
                               well_in=-1, well_out=-1, name=f"{p.name}_window{nx}x{ny}x{nz}")


MILLIDARCY = 9.869233e-16   # m^2

# Capillary-pressure parameter sets "Ex 1".."Ex 4" of Sec. 4 (Table of P_c
# parameters): (linear entry pressure P0, Brooks-Corey entry pressure Pd,
# Brooks-Corey lambda). Ex 1 is diffusion-dominated, Ex 2 advection-dominated,
# Ex 3 strongly advection-dominated.
PC_EXAMPLES = {1: (1e5, 1e6, 2.5), 2: (1e4, 1e5, 0.8), 3: (1e3, 2e4, 2.5), 4: (1e6, 1e6, 0.8)}

# time step [days] and number of steps of the gravity study per example
# (final times 20, 8 and 2 days)
GRAVITY_DT_DAYS = {1: 10.0, 2: 4.0, 3: 1.0}
GRAVITY_STEPS = 2


def config_gravity_2d(n: int, example: int = 1, pc_model: int = PC_BROOKS_COREY) -> Problem:
    """The gravity example of Sec. 4.2: a vertical 20 m x 20 m box (unit
    thickness, depth = y, so row iy = 0 is the top) on an n x n mesh,
    homogeneous 100 mD, water injected at 5 m^3/day into the top-left cell,
    outlet on the x = L face of the top-right cell. Fluids, porosity and the
    outlet state are those of the two-dimensional oil-water example (1000 /
    700 kg/m^3, 1 / 10 cP, phi 0.2, S_wr 0, outlet p_w = 0 and S_w = 0.2);
    the capillary model takes parameter set `example`."""
    k = np.full(n * n, 100.0 * MILLIDARCY)
    p0, pd, lam = PC_EXAMPLES[example]
    h = 20.0 / n
    return Problem(dim=2, nx=n, ny=n, nz=1, kx=k, ky=k.copy(), kz=k.copy(), hx=h, hy=h, hz=1.0,
                   phi=0.2, mu_w=1e-3, mu_n=1e-2, rho_w=1000.0, rho_n=700.0, g=9.81,
                   pc_model=pc_model, pc_p0=p0, pc_pd=pd, bc_lambda=lam, s_wr=0.0, s_nr=0.0,
                   u_in=0.0, p_out=0.0, sn_out=0.8, q_in=5.0 / DAY, well_in=0, well_out=n - 1,
                   name=f"2d_gravity_{n}x{n}_ex{example}_{'bc' if pc_model == PC_BROOKS_COREY else 'lin'}")


def config_oil_water_2d(example: int = 1, pc_model: int = PC_LINEAR, nx: int = 100, nz: int = 20,
                        sigma: float = 2.0, ell=(2.0, 16.0)) -> Problem:
    """The two-dimensional oil-water example of Sec. 4.1: a 762 m x 15.24 m
    vertical section (depth = the second coordinate) on a 100 x 20 mesh, the
    geometry of the SPE10 model-1 section, whose single cell layer across is
    7.62 m thick; the model's unit thickness carries the 50 m^3/day injected
    into the lower-left cell as 50 / 7.62 m^3/day per metre of thickness,
    outlet (p_w = 0, S_w = 0.2) on the x = L face of the top-right cell, no
    gravity, fluids and porosity of the table of input data, capillary
    parameter set `example`. The SPE10 permeability is not available; a
    seeded log-normal stand-in with sample std `sigma` of ln k, correlation
    lengths `ell` = (vertical, horizontal) in cells (layered, like the SPE10
    sections) and geometric mean 100 mD takes its place."""
    rng = _rng(6, nx, nz)
    lnk = lognormal_field((nz, nx), sigma, ell, np.log(100.0 * MILLIDARCY), rng)
    k = np.exp(lnk).reshape(-1)
    p0, pd, lam = PC_EXAMPLES[example]
    return Problem(dim=2, nx=nx, ny=nz, nz=1, kx=k, ky=k.copy(), kz=k.copy(), hx=762.0 / nx, hy=15.24 / nz,
                   hz=1.0, phi=0.2, mu_w=1e-3, mu_n=1e-2, rho_w=1000.0, rho_n=700.0, g=0.0,
                   pc_model=pc_model, pc_p0=p0, pc_pd=pd, bc_lambda=lam, s_wr=0.0, s_nr=0.0,
                   u_in=0.0, p_out=0.0, sn_out=0.8, q_in=50.0 / 7.62 / DAY, well_in=(nz - 1) * nx, well_out=nx - 1,
                   name=f"2d_oil_water_{nx}x{nz}_ex{example}_{'bc' if pc_model == PC_BROOKS_COREY else 'lin'}")


# the oil-water example runs 200 days in steps of 20 days
OIL_WATER_DT_DAYS = 20.0
OIL_WATER_STEPS = 10


def uniform_state(p: Problem, p_w: float = 1e5, s_n: float = 0.8) -> np.ndarray:
    """Uniform initial state (the oil-water examples of Sec. 4: p_w = 1e5 Pa,
    S_n = 0.8)."""
    u = np.empty(2 * p.ncell)
    u[0::2] = p_w
    u[1::2] = s_n
    return u


def cell_x(p: Problem) -> np.ndarray:
    """x coordinate of each cell centre, in cell order."""
    ix = np.arange(p.ncell) % p.nx
    return (ix + 0.5) * p.hx


def front_state(p: Problem, front_cells: float = None,
                s_init: float = 0.1, s_high: float = 0.9,
                dp: float = 3.2e4) -> Tuple[np.ndarray, np.ndarray]:
    """Deterministic linearisation state (u, u_old) with a saturation front.

    S_n(x) = s_init + (s_high - s_init) * (1 - tanh((x - x_f) / (2h))) / 2 with
    the front x_f a quarter of the way across; p_w falls linearly from
    p_out + dp at x = 0 to p_out at x = L. u_old is the same state with the
    front one cell further upstream. Both are interleaved (p_w, S_n) arrays.
    """
    L = p.nx * p.hx
    xf = L / 4.0 if front_cells is None else front_cells * p.hx
    x = cell_x(p)

    def sat(xf_):
        return s_init + (s_high - s_init) * 0.5 * (1.0 - np.tanh((x - xf_) / (2.0 * p.hx)))

    pres = p.p_out + dp * (1.0 - x / L)
    u = np.empty(2 * p.ncell)
    u[0::2] = pres
    u[1::2] = sat(xf)
    u_old = u.copy()
    u_old[1::2] = sat(xf - p.hx)
    return u, u_old


def initial_state(p: Problem, s_init: float = 0.1) -> np.ndarray:
    """Uniform start of a time-stepping run: p_w = p_out, S_n = s_init."""
    u = np.empty(2 * p.ncell)
    u[0::2] = p.p_out
    u[1::2] = s_init
    return u


def jitter(u: np.ndarray, seed: int, dp: float = 50.0, ds: float = 0.01) -> np.ndarray:
    """Seeded small perturbation of a state (breaks exact upwind ties)."""
    rng = _rng(99, seed)
    v = u.copy()
    v[0::2] += dp * rng.standard_normal(v.size // 2)
    v[1::2] += ds * rng.standard_normal(v.size // 2)
    return v


def poisson_2d(n: int):
    """5-point Laplacian (Dirichlet) on an n x n grid as CSR arrays (n^2 rows).

    Returned as (rowptr int32, col int32, val float64), columns ascending.
    """
    N = n * n
    rows, cols, vals = [], [], []
    for iy in range(n):
        for ix in range(n):
            i = ix + n * iy
            ent = []
            if iy > 0:
                ent.append((i - n, -1.0))
            if ix > 0:
                ent.append((i - 1, -1.0))
            ent.append((i, 4.0))
            if ix < n - 1:
                ent.append((i + 1, -1.0))
            if iy < n - 1:
                ent.append((i + n, -1.0))
            for c, v in ent:
                rows.append(i)
                cols.append(c)
                vals.append(v)
    return _coo_to_csr(N, rows, cols, vals)


def poisson_3d(n: int):
    """7-point Laplacian (Dirichlet) on an n^3 grid as CSR arrays."""
    N = n ** 3
    idx = np.arange(N)
    ix = idx % n
    iy = (idx // n) % n
    iz = idx // (n * n)
    rows = [idx]
    cols = [idx]
    vals = [np.full(N, 6.0)]
    for d, cond in ((-n * n, iz > 0), (-n, iy > 0), (-1, ix > 0),
                    (1, ix < n - 1), (n, iy < n - 1), (n * n, iz < n - 1)):
        r = idx[cond]
        rows.append(r)
        cols.append(r + d)
        vals.append(np.full(r.size, -1.0))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    return _coo_to_csr(N, r[order], c[order], v[order])


def poisson_1d(n: int):
    """tridiag(-1, 2, -1) of size n as CSR arrays."""
    rows, cols, vals = [], [], []
    for i in range(n):
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        rows.append(i); cols.append(i); vals.append(2.0)
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(-1.0)
    return _coo_to_csr(n, rows, cols, vals)


def _coo_to_csr(n, rows, cols, vals):
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int32)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return rowptr, cols, vals


def rhs_vector(n: int, seed: int) -> np.ndarray:
    """Seeded standard-normal right-hand side."""
    return _rng(7, seed).standard_normal(n)

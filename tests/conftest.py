import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger CPU oracle cases")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.lib()
    return O


@pytest.fixture(scope="session")
def inputs():
    from paper_1611_00127_gb300 import inputs as I
    return I


@pytest.fixture(scope="session")
def two_cell_cases(inputs):
    """The hand-derived two-cell flux cases of tests/golden/tpfa_two_cell.json
    as (case, Problem, u) triples; u is also the old state."""
    import json

    import numpy as np
    with open(os.path.join(os.path.dirname(__file__), "golden", "tpfa_two_cell.json")) as f:
        gold = json.load(f)
    com = gold["common"]
    out = []
    for c in gold["cases"]:
        g = c["grid"]
        along = np.asarray(g["k_along"], dtype=np.float64)
        across = np.asarray(g["k_across"], dtype=np.float64)
        if g["nz"] == 2:
            kx, ky, kz = across, across.copy(), along
        else:
            kx, ky, kz = along, across, across.copy()
        p = inputs.Problem(dim=g["dim"], nx=g["nx"], ny=g["ny"], nz=g["nz"], kx=kx, ky=ky, kz=kz,
                           phi=com["phi"], mu_w=com["mu_w"], mu_n=com["mu_n"], rho_w=com["rho_w"],
                           rho_n=com["rho_n"], g=com["g"], pc_model=com["pc_model"], pc_p0=com["pc_p0"],
                           bc_lambda=com["bc_lambda"], u_in=com["u_in"], p_out=com["p_out"],
                           sn_out=com["sn_out"], well_out=g["well_out"])
        u = np.empty(4)
        u[0::2] = c["pw"]
        u[1::2] = c["sn"]
        out.append((c, p, u))
    return out, com["dt"]

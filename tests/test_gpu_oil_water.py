"""The oil-water study (Sec. 4.1, Tables performance_q5_1..q5_3) on the GPU.

Ten 20-day backward-Euler steps of the 100 x 20 section with the linear and
the Brooks-Corey capillary models: for the (example, model, preconditioner)
cases the oracle converges in, the GPU time stepping (Newton with the
Appleyard chop, FGMRES, FP64 V-cycles) takes the oracle's Newton iteration
counts (within one per step) and linear counts (within 10 % per step), and
its state after every step matches the oracle's within the Newton tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1611_00127_gb300 import rsflow, studies
    rsflow.lib()
    return studies


ORACLE_KIND = {"AMG": (0, 0, 0), "CPR1": (1, 2, 1), "CPR2": (2, 2, 1), "BF": (3, 0, 0)}


@pytest.mark.parametrize("ex,model,kinds", [
    (1, 1, ("AMG", "CPR1", "CPR2", "BF")),
    (3, 1, ("CPR1", "CPR2")),
    (4, 1, ("AMG", "CPR1")),
    (1, 2, ("AMG", "CPR1", "CPR2", "BF")),
    (3, 2, ("AMG", "CPR1", "CPR2")),
])
def test_oil_water_steps_match_oracle(S, oracle, inputs, ex, model, kinds):
    p = inputs.config_oil_water_2d(ex, model)
    dt = inputs.OIL_WATER_DT_DAYS * inputs.DAY
    for kind in kinds:
        k, dec, p1 = ORACLE_KIND[kind]
        r = S.run_oil_water(ex, model, kind, keep_states=True)
        assert r["converged"], (ex, model, kind, r["steps"])
        u = inputs.uniform_state(p)
        for s in range(inputs.OIL_WATER_STEPS):
            u, st, ni, li, _ = oracle.newton(p, u, u, dt, oracle.NewtonParams(
                max_newton=40, max_ds=0.2, prec=oracle.PrecParams(kind=k, decouple=dec, p1=p1)))
            assert st == 0
            g = r["steps"][s]
            assert abs(g["ni"] - ni) <= 1, (ex, model, kind, s, g, ni)
            assert abs(g["li"] - li) <= max(2, 0.1 * li), (ex, model, kind, s, g, li)
            ug = r["states"][s]
            np.testing.assert_allclose(ug[1::2], u[1::2], atol=1e-5)
            np.testing.assert_allclose(ug[0::2], u[0::2], rtol=1e-5, atol=1e-5 * np.abs(u[0::2]).max())

"""Host-side logic of the study runner (no GPU): the preconditioner table
maps each study name to the C-ABI's kind, decoupling and first stage, the
Newton parameters carry the chop and tolerances the studies state, and the
report tables print LI/NI per case with '-' where a step did not converge."""
import pytest

pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    from paper_1611_00127_gb300 import studies
    return studies


def test_preconditioner_table(S):
    from paper_1611_00127_gb300 import rsflow as R
    assert S.KINDS["AMG"] == (R.AMG_J, R.DECOUPLE_NONE, R.P1_BLOCK_JACOBI)
    assert S.KINDS["CPR1"] == (R.CPR1, R.DECOUPLE_QIMPES, R.P1_ILU0)
    assert S.KINDS["CPR2"] == (R.CPR2, R.DECOUPLE_QIMPES, R.P1_ILU0)
    assert S.KINDS["BF"][0] == R.BF
    assert S.KINDS["CPR1_BJ"][2] == R.P1_BLOCK_JACOBI and S.KINDS["CPR2_BJ"][2] == R.P1_BLOCK_JACOBI
    assert S.MESHES == (20, 40, 80, 160)


def test_newton_parameters(S):
    from paper_1611_00127_gb300 import rsflow as R
    p = S.newton_params("CPR2", R.FP32, rtol=1e-8)
    assert p.max_ds == 0.2 and p.ftol == 1e-6 and p.max_newton == 40
    assert (p.gmres.m, p.gmres.maxit, p.gmres.rtol) == (30, 1000, 1e-8)
    assert (p.prec.kind, p.prec.decouple, p.prec.p1) == (R.CPR2, R.DECOUPLE_QIMPES, R.P1_ILU0)
    assert p.prec.amg.precision == R.FP32
    c = p.c()                      # the ctypes struct the C-ABI receives
    assert c.max_ds == 0.2 and c.prec.p1 == R.P1_ILU0 and c.gmres.maxit == 1000
    assert c.prec.amg.restriction == 0
    b = S.newton_params("BF", restriction=3).c()
    assert b.prec.kind == R.BF and b.prec.amg.restriction == 3 and b.prec.amg.precision == R.FP64


def test_report_tables(S):
    from paper_1611_00127_gb300 import inputs as I
    res = [dict(example=1, kind="AMG", n=20, converged=True, LI_per_NI=9.94),
           dict(example=1, kind="AMG", n=40, converged=False, LI_per_NI=12.0),
           dict(example=1, kind="BF", n=20, converged=True, LI_per_NI=21.2)]
    t = S.table(res, 1, ["AMG", "BF"], [20, 40]).splitlines()
    assert t[0].startswith("Ex 1 (dt = 10 days)")
    assert t[1].split()[1:] == ["9.9", "-"]
    assert t[2].split()[1:] == ["21.2", "-"]          # no run at 40^2
    ow = [dict(example=2, kind="CPR1", pc_model=I.PC_LINEAR, converged=True, NI=76, LI=1370, LI_per_NI=18.03),
          dict(example=2, kind="CPR1", pc_model=I.PC_BROOKS_COREY, converged=False, NI=3, LI=900, LI_per_NI=300.0)]
    t = S.oil_water_table(ow, ["CPR1"], [2], [I.PC_LINEAR, I.PC_BROOKS_COREY]).splitlines()
    assert "linear" in t[0] and "Brooks-Corey" in t[0]
    assert t[1].split() == ["CPR1", "76", "1370", "18.0", "-"]

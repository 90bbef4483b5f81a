"""jacobian_assemble_noalloc, the assembly entry point that allocates no
device memory (for callers that cannot call cudaMalloc), against the
allocating jacobian_assemble through the C-ABI.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test. It must pass alone in a fresh process and
after the other tests (the library's fixed arrays keep the previous call's
contents, and every call overwrites them).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1611_00127_gb300 import rsflow
    rsflow.lib()
    return rsflow


def _assemble_both(R, inputs, probs, states):
    dp = R.DeviceProblems(probs)
    u = torch.as_tensor(np.concatenate([s[0] for s in states]), device="cuda")
    uo = torch.as_tensor(np.concatenate([s[1] for s in states]), device="cuda")
    Ja, Jb = R.Bsr2.pattern(dp), R.Bsr2.pattern(dp)
    Fa = torch.empty(2 * dp.ncell, dtype=torch.float64, device="cuda")
    Fb = torch.full_like(Fa, float("nan"))
    Jb.val.fill_(float("nan"))
    R.jacobian_assemble(dp, u, uo, inputs.DAY, Ja, Fa)
    R.jacobian_assemble_noalloc(dp, u, uo, inputs.DAY, Jb, Fb)
    torch.cuda.synchronize()
    return (Fa.cpu().numpy(), Ja.val.cpu().numpy()), (Fb.cpu().numpy(), Jb.val.cpu().numpy())


def _check_equal(a, b):
    (Fa, Ja), (Fb, Jb) = a, b
    np.testing.assert_allclose(Fb, Fa, rtol=1e-12, atol=1e-14 * np.abs(Fa).max())
    np.testing.assert_allclose(Jb, Ja, rtol=1e-12, atol=1e-14 * np.abs(Ja).max())


def test_noalloc_assembly_matches_allocating_call_twice(R, inputs):
    # first call: one 2D grid at a front state
    p1 = inputs.config_small_2d()
    a, b = _assemble_both(R, inputs, [p1], [inputs.front_state(p1)])
    _check_equal(a, b)
    # second call in a row: a batch of a 3D grid and a log-normal 2D grid,
    # different sizes, so the fixed arrays are reused with new contents
    rng = np.random.default_rng(2)
    k = np.exp(rng.normal(np.log(1e-12), 1.0, 9 * 7 * 5))
    p2 = inputs.Problem(dim=3, nx=9, ny=7, nz=5, kx=k, ky=k, kz=0.1 * k, pc_model=2, pc_pd=5e3, g=9.81)
    p3 = inputs.config_lognormal_2d(1e4, n=40)
    s2 = inputs.front_state(p2)
    s2 = (inputs.jitter(s2[0], 4), s2[1])
    a, b = _assemble_both(R, inputs, [p2, p3], [s2, inputs.front_state(p3)])
    _check_equal(a, b)


def test_noalloc_rejects_sizes_beyond_its_limit(R, inputs):
    p = inputs.homogeneous(300, 300)           # 90000 cells > 65536
    dp = R.DeviceProblems(p)
    u = torch.zeros(2 * p.ncell, dtype=torch.float64, device="cuda")
    F = torch.empty_like(u)
    with pytest.raises(R.RsError, match="exceed the limit of 65536"):
        R.jacobian_assemble_noalloc(dp, u, u, inputs.DAY, None, F)

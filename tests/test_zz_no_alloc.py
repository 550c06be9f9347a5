"""The entry point that allocates nothing, against the regular entry point.

subapsnap_solve_batch_xhat_noalloc serves callers that cannot allocate device
memory when they solve (a framework that reserved all device memory up front,
or a latency-critical loop where an allocation would synchronise the device).
It stages the coefficient vectors in a fixed device array instead of a
context-owned buffer.  This test calls it through the C ABI twice in a row,
with different parameters, and checks both outputs against
subapsnap_solve_batch with SAS_OUT_XHAT, within the plain float64 parity
tolerance used elsewhere (1e-10 relative per parameter), and against the CPU
oracle's x_hat at the same tolerance, so that a fault shared by both entry
points does not pass unseen.  On a fresh context it calls the entry point
before any regular solve and checks that the device's free memory does not
change around the call; a mixed-mode context (whose regular x_hat comes from
other kernels) gets the same oracle comparison.  It also checks that a batch
larger than the fixed array is refused.  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import online  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver  # noqa: E402
from workloads import get_config  # noqa: E402
from workloads import snapshots as wsnap  # noqa: E402


def _rows_rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_noalloc_matches_solve_batch_twice():
    prob = get_config("diffusion_2d", N=40, r=30, s=60, m=500)
    S = wsnap.basis(prob)
    rng = np.random.default_rng(3)
    J = np.sort(rng.choice(prob.n, prob.s, replace=False))
    solver = AffineSolver(prob, S, J, mode=api.SAS_MODE_PLAIN, device="cuda")
    batches = [prob.test_params[:200], prob.test_params[200:437]]  # two calls, different sizes
    for params in batches:
        m = params.shape[0]
        assert m * prob.r <= api.SAS_NOALLOC_MAX_Y
        P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
        ref = torch.empty((m, prob.n), dtype=torch.float64, device="cuda")
        rho_ref = torch.empty(m, dtype=torch.float64, device="cuda")
        api.subapsnap_solve_batch(solver.ctx, P, m, api.SAS_OUT_XHAT, ref, None, rho_ref)
        out = torch.full((m, prob.n), float("nan"), dtype=torch.float64, device="cuda")
        rho = torch.empty(m, dtype=torch.float64, device="cuda")
        api.subapsnap_solve_batch_xhat_noalloc(solver.ctx, P, m, out, None, rho)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert _rows_rel(a, b).max() <= 1e-10
        np.testing.assert_allclose(rho.cpu().numpy(), rho_ref.cpu().numpy(), rtol=1e-12, atol=0)
        Yo, _ = online.solve_many(prob, S, J, params[:8])
        assert _rows_rel(a[:8], Yo @ S.T).max() <= 1e-10
    # a batch beyond the fixed array is refused before any work
    m_big = api.SAS_NOALLOC_MAX_Y // prob.r + 1
    P = torch.zeros((m_big, prob.dp), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(api.SasError) as ei:
        api.subapsnap_solve_batch_xhat_noalloc(solver.ctx, P, m_big, out)
    assert ei.value.code == api.SAS_EINVAL
    solver.close()


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED], ids=["plain", "mixed"])
def test_noalloc_first_call_allocates_nothing(mode):
    """A fresh context: the no-allocation call comes before any regular solve (so no
    scratch the regular path grows can serve it), the device's free memory is the
    same before and after it, and its x_hat matches the oracle's."""
    prob = get_config("diffusion_2d", N=32, r=20, s=40, m=64)
    S = wsnap.basis(prob)
    J = np.sort(np.random.default_rng(4).choice(prob.n, prob.s, replace=False))
    solver = AffineSolver(prob, S, J, mode=mode, device="cuda")
    params = prob.test_params
    m = params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    out = torch.full((m, prob.n), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    api.subapsnap_solve_batch_xhat_noalloc(solver.ctx, P, m, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    Yo, _ = online.solve_many(prob, S, J, params)
    assert _rows_rel(out.cpu().numpy(), Yo @ S.T).max() <= 1e-10
    solver.close()

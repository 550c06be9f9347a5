"""The entry point that allocates nothing, against the regular entry point.

subapsnap_solve_batch_xhat_noalloc serves callers that cannot allocate device
memory when they solve (a framework that reserved all device memory up front,
or a latency-critical loop where an allocation would synchronise the device).
It stages the coefficient vectors in a fixed device array instead of a
context-owned buffer.  This test calls it through the C ABI twice in a row,
with different parameters, and checks both outputs against
subapsnap_solve_batch with SAS_OUT_XHAT, within the plain float64 parity
tolerance used elsewhere (1e-10 relative per parameter).  It also checks that
a batch larger than the fixed array is refused.  The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

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
    # a batch beyond the fixed array is refused before any work
    m_big = api.SAS_NOALLOC_MAX_Y // prob.r + 1
    P = torch.zeros((m_big, prob.dp), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(api.SasError) as ei:
        api.subapsnap_solve_batch_xhat_noalloc(solver.ctx, P, m_big, out)
    assert ei.value.code == api.SAS_EINVAL
    solver.close()

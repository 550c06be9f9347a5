"""Persistent batched launch over operator families of uneven s and r.

A multi-problem plan solves three contexts (different n, r, s, K) in one launch,
optionally replayed from a CUDA graph.  Each parameter runs the same per-task
solve as subapsnap_solve_batch with the same launch shape: plain float64 outputs
must be bit-identical to the per-context solves; mixed outputs (a float32 body
the compiler may contract differently in another kernel, then refined to float64
accuracy) within 1e-9.  Both are also checked against the oracle (mixed: the
conditioning bound of the refined float32 solve).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver  # noqa: E402

from _problems import Case, mixed_bound  # noqa: E402


@pytest.fixture(scope="module")
def cases():
    return [Case("reaction_diffusion_1d", n=700, r=12, s=24, m=257),
            Case("diffusion_2d", N=30, r=40, s=80, m=130),
            Case("diffusion_2d", basis="random", N=24, r=20, s=50, m=61, seed_basis=3)]


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED])
def test_multi_plan_matches_single_solves(cases, mode):
    solvers = [AffineSolver(c.prob, c.S, c.J, mode=mode, device="cuda") for c in cases]
    params = [torch.from_numpy(np.ascontiguousarray(c.prob.test_params)).cuda() for c in cases]
    ref, outs, rhos, flags = [], [], [], []
    for sv, P, c in zip(solvers, params, cases):
        y = torch.empty((P.shape[0], c.prob.r), dtype=torch.float64, device="cuda")
        sv.solve(P, api.SAS_OUT_Y, y)
        ref.append(y)
        outs.append(torch.full_like(y, float("nan")))
        rhos.append(torch.empty(P.shape[0], dtype=torch.float64, device="cuda"))
        flags.append(torch.zeros(P.shape[0], dtype=torch.int32, device="cuda"))
    plan = api.subapsnap_multi_plan_create([s.ctx for s in solvers], params, api.SAS_OUT_Y, outs, flags, rhos)
    for use_graph in (False, True, True):
        for o in outs:
            o.fill_(float("nan"))
        api.subapsnap_multi_plan_launch(plan, use_graph)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            if mode == api.SAS_MODE_PLAIN:
                assert torch.equal(o, r)
            else:
                # the float32 body inlined into another kernel may contract differently;
                # both answers are refined to float64 accuracy of the same system
                rel = (torch.linalg.vector_norm(o - r, dim=1) / torch.linalg.vector_norm(r, dim=1)).max()
                assert rel.item() <= 1e-9, rel.item()
    for c, o in zip(cases, outs):
        Yo, rho_o = c.oracle_solve(c.prob.test_params[:20])
        err = np.linalg.norm(o[:20].cpu().numpy() - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
        if mode == api.SAS_MODE_PLAIN:
            assert err.max() <= 1e-10
        else:
            # the refined float32 solve converges to the LS solution of the
            # float32-perturbed matrix: bounded per parameter by its conditioning
            bound = mixed_bound(c.prob, c.S, c.J, c.prob.test_params[:20], Yo, rho_o)
            assert (err <= bound).all(), (err.max(), bound.min())
    api.subapsnap_multi_plan_destroy(plan)
    for s in solvers:
        s.close()

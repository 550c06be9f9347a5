"""Parity at the benchmark's full size, in the launch configuration bench.py times.

2-D diffusion on the 1024 x 1024 grid (n = 1,048,576), r = 60, s = 120, the
4096 test parameters solved in chunks of 256 with x_hat output.  The oracle
cannot reconstruct every x_hat, so it is compared on sampled outputs it can
compute one by one:
  * J from the device CPQR against the oracle's CPQR rounds (float64 pivot
    rule; near-ties are reported instead of compared);
  * y for 12 parameters spread over the batch (plain: 1e-10 relative;
    mixed: the refinement bound of tests/_problems.mixed_bound);
  * x_hat at 4096 sampled rows of those parameters (plain: 1e-10 relative to
    ||x||_inf; mixed, float64 from the tensor-core digit products: 1e-10 too);
  * the subsampled residual, within the rounding of the assembly itself
    (estimated from two float64 assemblies on the host);
  * properties that hold at any size for the whole batch: finite outputs, no
    ill-conditioning flags.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import online, problem as oproblem, selection  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver, csr_to_device, select_rows  # noqa: E402
from workloads import get_config  # noqa: E402
from workloads import snapshots as wsnap  # noqa: E402

from _problems import mixed_bound  # noqa: E402

CHUNK = 256


@pytest.fixture(scope="module")
def full():
    prob = get_config("diffusion_2d")  # N = 1024, r = 60, s = 120, m = 4096
    blocks = [csr_to_device(A, "cuda") for A in prob.blocks]
    S_rows, res = wsnap.diffusion_basis_torch(prob, device="cuda")
    assert res.max() < 1e-9
    J, gaps = select_rows(prob, S_rows, blocks, prob.sel_param, prob.s)
    S = S_rows.cpu().numpy().T.copy()
    return prob, blocks, S_rows, S, J, gaps


def test_fullsize_row_selection(full):
    prob, blocks, S_rows, S, J, gaps = full
    V = np.asarray(oproblem.full_matrix(prob, prob.sel_param) @ S)
    Jo, gaps_o = selection.cpqr_rows(V, prob.s)
    near = np.nonzero(gaps_o < 1e-10)[0]
    upto = near[0] if near.size else prob.s
    print(f"full-size J: first near-tie at step {upto if near.size else None}, min gap {gaps_o.min():.2e}")
    np.testing.assert_array_equal(J[:upto], Jo[:upto])


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED])
def test_fullsize_sampled_outputs(full, mode):
    prob, blocks, S_rows, S, J, gaps = full
    solver = AffineSolver(prob, None, J, mode=mode, device="cuda", S_device=S_rows,
                          blocks_device=blocks)
    m, n = prob.test_params.shape[0], prob.n
    P = torch.from_numpy(np.ascontiguousarray(prob.test_params)).cuda()
    rng = np.random.default_rng(4)
    pick = np.unique(np.concatenate([[0, CHUNK - 1, CHUNK, m - 1], rng.choice(m, 8, replace=False)]))
    rows = np.sort(rng.choice(n, 4096, replace=False))
    rows_t = torch.from_numpy(rows).cuda()
    out = torch.empty((CHUNK, n), dtype=torch.float64, device="cuda")
    flags = torch.zeros(m, dtype=torch.int32, device="cuda")
    rho = torch.empty(m, dtype=torch.float64, device="cuda")
    sampled = {}
    for c in range(m // CHUNK):
        sl = slice(c * CHUNK, (c + 1) * CHUNK)
        solver.solve(P[sl], api.SAS_OUT_XHAT, out, flags[sl], rho[sl])
        for j in pick[(pick >= sl.start) & (pick < sl.stop)]:
            sampled[int(j)] = out[j - sl.start].index_select(0, rows_t).double().cpu().numpy()
        assert torch.isfinite(out).all().item()
    Y = torch.empty((m, prob.r), dtype=torch.float64, device="cuda")
    solver.solve(P, api.SAS_OUT_Y, Y)
    torch.cuda.synchronize()
    Y = Y.cpu().numpy()
    flags = flags.cpu().numpy()
    rho = rho.cpu().numpy()
    assert not (flags & (api.SAS_FLAG_ILLCOND | api.SAS_FLAG_NONFINITE)).any()
    worst_y, worst_x, worst_ratio = 0.0, 0.0, 0.0
    for j in pick:
        yo, rho_o = online.solve_one(prob, S, J, prob.test_params[j])
        ey = np.linalg.norm(Y[j] - yo) / np.linalg.norm(yo)
        if mode == api.SAS_MODE_MIXED:
            bound = mixed_bound(prob, S, J, prob.test_params[j:j + 1], [yo], [rho_o])[0]
            worst_ratio = max(worst_ratio, ey / bound)
        xo = S[rows] @ yo
        ex = np.abs(sampled[j] - xo).max() / np.abs(S @ yo).max()
        worst_y, worst_x = max(worst_y, ey), max(worst_x, ex)
        # rho is sensitive to the rounding of the assembly (each row of A_J S
        # cancels terms of size h^-2 |S|): bound |d rho| by the discrepancy between
        # two float64 assemblies computed here (explicit rows vs sum_k theta_k G_k)
        th = np.concatenate([[1.0], prob.test_params[j]])
        M_rows = online.subsampled_matrix(prob, S, J, prob.test_params[j])
        M_aff = sum(t * np.asarray(A[J] @ S) for t, A in zip(th, prob.blocks))
        dM = np.linalg.norm(M_rows - M_aff, 2) + 1.1e-16 * np.linalg.norm(M_rows, 2)
        tol_rho = 1e-6 * rho_o + 8 * dM * np.linalg.norm(yo) / np.linalg.norm(prob.b[J])
        assert abs(rho[j] - rho_o) <= tol_rho, (rho[j], rho_o, tol_rho)
    print(f"full-size mode {mode}: max rel err y {worst_y:.2e}, x_hat sampled {worst_x:.2e}")
    if mode == api.SAS_MODE_PLAIN:
        assert worst_y <= 1e-10 and worst_x <= 1e-10
    else:
        assert worst_ratio <= 1.0 and worst_x <= 1e-10
    solver.close()

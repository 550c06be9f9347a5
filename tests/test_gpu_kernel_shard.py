"""Kernel rows split over point shards (the multi-GPU split of the Gaussian-kernel rows over N).

Each shard's context holds a block of the points and forms the partial rows
M_g = K_sigma(X_J, X_g) S_g, plus lambda S_J on the one shard that owns that term.  The
sum over the shards is the full M, and any shard's context solves the least squares from
it.  Here the shards run one after the other on one GPU (no kernel waits on another), and
the sum stands in for the all-reduce:
  * the summed rows equal the full context's rows (plain: float64 up to the reordered sums
    over the points; mixed: entry by entry within twice the tensor-core rows' error bound,
    relative to sum_j |K_ij| |S_jl|);
  * y solved from the summed rows equals the full context's y (plain: 1e-10 relative where
    kappa(M) u <= 1e-11; mixed: the kernel-row test's bound 4 kappa 64 u_32);
  * shards of unequal size and a shard of a single point;
  * a shard context refuses subapsnap_solve_batch (its own rows are partial).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import krr, selection  # noqa: E402
from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import KernelShard, KernelSolver  # noqa: E402
from workloads import get_config  # noqa: E402
from workloads import snapshots as wsnap  # noqa: E402

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def case():
    prob = get_config("kernel_ridge", N=2500, r=16, s=48, m=40)
    S = wsnap.basis(prob)
    V = krr.full_matrix(prob.X, prob.sel_param) @ S
    J, _ = selection.cpqr_rows(V, prob.s)
    return prob, S, J


def device_arrays(prob, S):
    X = torch.from_numpy(np.ascontiguousarray(prob.X)).cuda()
    Sd = torch.from_numpy(np.ascontiguousarray(S.T)).cuda()  # (r, N): column-major N x r
    b = torch.from_numpy(np.ascontiguousarray(prob.b)).cuda()
    return X, Sd, b


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED], ids=["plain", "mixed"])
@pytest.mark.parametrize("world", [2, 3])
def test_shard_rows_sum_to_the_full_rows_and_solve(case, mode, world):
    prob, S, J = case
    X, Sd, b = device_arrays(prob, S)
    params = np.ascontiguousarray(prob.test_params)
    m, s, r = params.shape[0], prob.s, prob.r
    P = torch.from_numpy(params).cuda()
    full = KernelSolver(prob, S, J, mode=mode, device="cuda", S_device=Sd, X_device=X, b_device=b)
    Mfull = torch.empty((m, r, s), dtype=torch.float64, device="cuda")  # block q: column-major s x r
    api.subapsnap_kernel_rows(full.ctx, P, m, Mfull)
    Yfull = torch.empty((m, r), dtype=torch.float64, device="cuda")
    full.solve(P, api.SAS_OUT_Y, Yfull)
    shards = [KernelShard.from_full(X, Sd, b, J, g, world, r, mode) for g in range(world)]
    Msum = torch.zeros_like(Mfull)
    part = torch.empty_like(Mfull)
    for sh in shards:
        sh.rows(P, part)
        Msum += part  # stands in for the all-reduce over the ranks
    Y = torch.empty((m, r), dtype=torch.float64, device="cuda")
    rho = torch.empty(m, dtype=torch.float64, device="cuda")
    shards[world - 1].solve_rows(P, Msum, Y, None, rho)
    torch.cuda.synchronize()
    Mf, Ms = Mfull.cpu().numpy(), Msum.cpu().numpy()
    dm = np.array([np.abs(Ms[q] - Mf[q]).max() / np.abs(Mf[q]).max() for q in range(m)])
    Yo, rho_o = krr.solve_many(prob, S, J, params)
    kap = np.array([np.linalg.cond(krr.subsampled_matrix(prob.X, S, J, p)) for p in params])
    Yd, Yf = Y.cpu().numpy(), Yfull.cpu().numpy()
    err_full = np.linalg.norm(Yd - Yf, axis=1) / np.linalg.norm(Yf, axis=1)
    err_o = np.linalg.norm(Yd - Yo, axis=1) / np.linalg.norm(Yo, axis=1)
    print(f"{world} shards, mode {mode}: rows rel diff max {dm.max():.1e}, y vs full {err_full.max():.1e}, "
          f"y vs oracle {err_o.max():.1e} (kappa max {kap.max():.1e})")
    if mode == api.SAS_MODE_PLAIN:
        assert dm.max() <= 1e-13
        strict = kap * 1.1e-16 <= 1e-11
        assert strict.sum() > 0 and err_o[strict].max() <= 1e-10
        assert (np.abs(rho.cpu().numpy() - rho_o) <= 1e-8 * rho_o + 64 * kap * 1.1e-16).all()
    else:
        # each side carries the tensor-core rows' error: ~3 x 2^-21 per split product and the
        # float32 accumulation of a 1024-point segment, both relative to sum_j |K_ij| |S_jl|
        # (not to |M|, which cancels); the shards place the segment boundaries differently
        for q, (sigma, lam) in enumerate(params):
            absM = krr.kernel_rows(prob.X, J, sigma) @ np.abs(S) + lam * np.abs(S[J])  # s x r
            dq = np.abs(Ms[q].T - Mf[q].T)
            assert (dq <= 2 * (3 * 2.0 ** -21 + 1024 * U32) * absM + 1e-300).all(), q
        assert (err_o <= 4 * kap * 64 * U32 + 1e-10).all()
    for sh in shards:
        sh.close()
    full.close()


def test_uneven_shards_and_a_single_point_shard(case):
    prob, S, J = case
    X, Sd, b = device_arrays(prob, S)
    params = np.ascontiguousarray(prob.test_params[:8])
    m, s, r, n = params.shape[0], prob.s, prob.r, prob.n
    P = torch.from_numpy(params).cuda()
    Jd = torch.as_tensor(np.asarray(J), device="cuda")
    XJ, SJ, bJ = X.index_select(0, Jd).contiguous(), Sd.index_select(1, Jd).contiguous(), b.index_select(0, Jd)
    cuts = [(0, 1), (1, 1000), (1000, n)]  # a single point, then two uneven blocks
    Msum = torch.zeros((m, r, s), dtype=torch.float64, device="cuda")
    part = torch.empty_like(Msum)
    shards = [KernelShard(X, Sd, XJ, SJ, bJ.contiguous(), slice(a, c), r, s, owns_lambda=(a == 0))
              for a, c in cuts]
    for sh in shards:
        sh.rows(P, part)
        Msum += part
    torch.cuda.synchronize()
    Mo = np.stack([krr.subsampled_matrix(prob.X, S, J, p) for p in params])  # m x s x r
    Ms = np.transpose(Msum.cpu().numpy(), (0, 2, 1))
    assert np.abs(Ms - Mo).max() <= 1e-13 * np.abs(Mo).max()
    with pytest.raises(api.SasError) as ei:
        api.subapsnap_solve_batch(shards[0].ctx, P, m, api.SAS_OUT_Y,
                                  torch.empty((m, r), dtype=torch.float64, device="cuda"))
    assert ei.value.code == api.SAS_ENOTSUP
    for sh in shards:
        sh.close()

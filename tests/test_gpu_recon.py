"""Mixed-form float32 reconstruction (SAS_OPT_XHAT_F32 = 1) on the tensor cores
(tcgen05) against the oracle.

x_hat in float32 from tf32 splits of S and y: three products, relative
error ~2^-21 per product, so <= 2e-6 relative per parameter is the bound.
Shapes cover ragged row tiles (n not a multiple of 128), ragged parameter
tiles (m not a multiple of 64), one and two K boxes (r <= 32, r <= 64),
the tf32 forms (64- and 128-parameter tiles) and the f16 form (S and y in
power-of-two-scaled f16 hi / 2^11 lo splits, three products),
the split of a row tile's parameter tiles into ranges (fewer row tiles than
SMs) and units that stream many parameter tiles past one resident S tile.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver  # noqa: E402

from _problems import Case  # noqa: E402


def xhat(case, kernel, params, on_device=False, store=0):
    solver = AffineSolver(case.prob, case.S, case.J, mode=api.SAS_MODE_MIXED, device="cuda")
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_XHAT_F32, 1)
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_RECON_KERNEL, kernel)
    api.subapsnap_set_option(solver.ctx, api.SAS_OPT_RECON_STORE, store)
    m = params.shape[0]
    P = torch.from_numpy(np.ascontiguousarray(params)).cuda()
    out = torch.full((m, case.prob.n), float("nan"), dtype=torch.float32, device="cuda")
    solver.solve(P, api.SAS_OUT_XHAT, out)
    st = api.subapsnap_device_status(solver.ctx)
    torch.cuda.synchronize()
    solver.close()
    assert st == 0
    if on_device:
        return out
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,r,s,m", [(45, 60, 120, 300), (40, 20, 40, 130), (32, 64, 128, 128),
                                     (48, 33, 70, 1), (20, 60, 120, 1000), (12, 30, 60, 777)])
def test_tensor_core_reconstruction(N, r, s, m):
    case = Case("diffusion_2d", basis="random", N=N, r=r, s=s, m=m)
    params = case.prob.test_params
    Yo, _ = case.oracle_solve(params)
    Xo = Yo @ case.S.T
    Xcc = xhat(case, 1, params)
    e_cc = np.linalg.norm(Xcc - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
    assert e_cc.max() <= 2e-6
    # tf32 64- and 128-parameter tiles, f16 splits; TMA-store and direct-store epilogues
    for kernel, store in ((2, 0), (3, 0), (5, 0), (5, 1), (3, 1), (6, 1), (0, 1)):
        Xtc = xhat(case, kernel, params, store=store)
        assert np.isfinite(Xtc).all()
        e_tc = np.linalg.norm(Xtc - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
        print(f"N={N} r={r} m={m}: tcgen05 ({kernel}, store {store}) max rel err {e_tc.max():.2e}, "
              f"CUDA cores {e_cc.max():.2e}")
        assert e_tc.max() <= 2e-6


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED, "mixed-f32"])
def test_reconstruct_entry_point_matches_solve(mode):
    """subapsnap_reconstruct(Y) gives the x_hat that solve_batch(SAS_OUT_XHAT) gives."""
    case = Case("diffusion_2d", basis="random", N=36, r=60, s=120, m=300)
    p = case.prob
    f32 = mode == "mixed-f32"
    solver = AffineSolver(p, case.S, case.J, mode=api.SAS_MODE_MIXED if f32 else mode, device="cuda")
    if f32:
        api.subapsnap_set_option(solver.ctx, api.SAS_OPT_XHAT_F32, 1)
    P = torch.from_numpy(np.ascontiguousarray(p.test_params)).cuda()
    m = P.shape[0]
    odt = torch.float32 if f32 else torch.float64
    X1 = torch.empty((m, p.n), dtype=odt, device="cuda")
    solver.solve(P, api.SAS_OUT_XHAT, X1)
    Y = torch.empty((m, p.r), dtype=torch.float64, device="cuda")
    solver.solve(P, api.SAS_OUT_Y, Y)
    X2 = torch.empty((m, p.n), dtype=odt, device="cuda")
    for c0 in range(0, m, 128):  # chunked, with a ragged last chunk
        solver.reconstruct(Y[c0:c0 + 128], X2[c0:c0 + 128])
    torch.cuda.synchronize()
    a, b = X2.double().cpu().numpy(), X1.double().cpu().numpy()
    err = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    assert err.max() <= (2e-6 if f32 else 1e-12)
    solver.close()


def test_tensor_core_reconstruction_large_n_many_batch_sizes():
    """n = 262,144 rows (2048 row tiles) with batch sizes that leave the last
    parameter tile full, partial or alone: the tcgen05 path against the CUDA-core
    path (both float32 from the same splits) and against the oracle on samples."""
    case = Case("diffusion_2d", basis="random", rows="random", N=512, r=60, s=120, m=300)
    p = case.prob
    for m in (1, 64, 100, 128, 256, 300):
        params = p.test_params[:m]
        Xcc = xhat(case, 1, params)
        for kernel, store in ((2, 0), (3, 0), (5, 0), (5, 1), (3, 1), (6, 1)):
            Xtc = xhat(case, kernel, params, store=store)
            d = np.linalg.norm(Xtc - Xcc, axis=1) / np.linalg.norm(Xcc, axis=1)
            bad = np.nonzero(d > 2e-6)[0]
            assert bad.size == 0, (kernel, store, m, bad[:8], d.max())
        Yo, _ = case.oracle_solve(params[:3])
        Xo = Yo @ case.S.T
        e = np.linalg.norm(Xtc[:3] - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
        assert e.max() <= 2e-6, (m, e)


def test_tensor_core_reconstruction_long_units():
    """n = 262,144 (2048 row tiles, more than the SMs: every unit streams all
    parameter tiles past its S tile) with m = 2100 (33 parameter tiles, the last
    ragged): tcgen05 against the CUDA-core path on the device, the oracle on samples."""
    case = Case("diffusion_2d", basis="random", rows="random", N=512, r=60, s=120, m=2100)
    p = case.prob
    params = p.test_params
    Xcc = xhat(case, 1, params, on_device=True)
    pick = [0, 63, 64, 1000, 2047, 2048, 2099]
    Yo, _ = case.oracle_solve(params[pick])
    Xo = Yo @ case.S.T
    for kernel in (3, 2, 5, 6):
        Xtc = xhat(case, kernel, params, on_device=True)
        assert torch.isfinite(Xtc).all().item()
        d = (torch.linalg.vector_norm(Xtc - Xcc, dim=1) / torch.linalg.vector_norm(Xcc, dim=1)).cpu().numpy()
        assert d.max() <= 2e-6, (kernel, np.argmax(d), d.max())
        Xs = Xtc[pick].double().cpu().numpy()
        e = np.linalg.norm(Xs - Xo, axis=1) / np.linalg.norm(Xo, axis=1)
        assert e.max() <= 2e-6, (kernel, e)
        del Xtc

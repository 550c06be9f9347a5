"""The host-buffer entry point gives what the device one gives, bit for bit.

subapsnap_solve_batch_host copies the parameters in, runs the same kernels and
brings the outputs back; x_hat lands directly in page-locked memory (the
reconstruction stores through the host mapping) or through device chunks for
pageable memory.  Either way every output equals subapsnap_solve_batch's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect with -m "not gpu"
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2510_04825_gb300 import api  # noqa: E402
from paper_2510_04825_gb300.solver import AffineSolver  # noqa: E402

from _problems import Case  # noqa: E402

DEV = "cuda"


@pytest.fixture(scope="module")
def c2d():
    return Case("diffusion_2d", N=40, r=20, s=40, m=70)


@pytest.fixture(scope="module")
def ctf():
    return Case("transfer_function", N=7, r=12, s=30, m=33)


def _device_reference(sv, P, kind, shape, dtype):
    out = torch.empty(shape, dtype=dtype, device=DEV)
    flags = torch.zeros(shape[0], dtype=torch.int32, device=DEV)
    rho = torch.empty(shape[0], dtype=torch.float64, device=DEV)
    sv.solve(P, kind, out, flags, rho)
    torch.cuda.synchronize()
    return out.cpu(), flags.cpu(), rho.cpu()


@pytest.mark.parametrize("mode", [api.SAS_MODE_PLAIN, api.SAS_MODE_MIXED, "mixed-f32"],
                         ids=["plain", "mixed", "mixed-f32"])
@pytest.mark.parametrize("pinned", [True, False, "chunked"], ids=["pinned", "pageable", "pageable-chunks"])
def test_host_buffers_match_device_buffers(c2d, mode, pinned):
    p = c2d.prob
    f32 = mode == "mixed-f32"
    sv = AffineSolver(p, c2d.S, c2d.J, mode=api.SAS_MODE_MIXED if f32 else mode, device=DEV)
    if f32:
        api.subapsnap_set_option(sv.ctx, api.SAS_OPT_XHAT_F32, 1)
    if pinned == "chunked":  # pageable x_hat through 17-parameter chunks, the last one ragged
        api.subapsnap_set_option(sv.ctx, api.SAS_OPT_HOST_CHUNK, 17 * p.n * 8)
        pinned = False
    params = np.ascontiguousarray(p.test_params)
    m = params.shape[0]
    P = torch.from_numpy(params).to(DEV)
    xdt = torch.float32 if f32 else torch.float64
    for kind, shape, dt in ((api.SAS_OUT_Y, (m, p.r), torch.float64), (api.SAS_OUT_XHAT, (m, p.n), xdt)):
        ref, fref, rref = _device_reference(sv, P, kind, shape, dt)
        out = torch.full(shape, float("nan"), dtype=dt)
        flags = torch.full((m,), -1, dtype=torch.int32)
        rho = torch.empty(m, dtype=torch.float64)
        hp = torch.from_numpy(params)
        if pinned:
            out, flags, rho, hp = out.pin_memory(), flags.pin_memory(), rho.pin_memory(), hp.pin_memory()
        api.subapsnap_solve_batch_host(sv.ctx, hp, m, kind, out, flags, rho)
        assert torch.equal(out, ref)
        assert torch.equal(flags, fref) and torch.equal(rho, rref)
    sv.close()


def test_host_buffers_complex_qoi_and_errors(ctf):
    p = ctf.prob
    sv = AffineSolver(p, ctf.S, ctf.J, mode=api.SAS_MODE_MIXED, device=DEV)
    params = np.ascontiguousarray(p.test_params)
    m = params.shape[0]
    ref, _, rref = _device_reference(sv, torch.from_numpy(params).to(DEV), api.SAS_OUT_QOI, (m,), torch.complex128)
    out = np.empty(m, dtype=np.complex128)
    rho = np.empty(m)
    api.subapsnap_solve_batch_host(sv.ctx, params, m, api.SAS_OUT_QOI, out, None, rho)
    np.testing.assert_array_equal(out, ref.numpy())
    np.testing.assert_array_equal(rho, rref.numpy())
    dev = torch.empty(m, dtype=torch.complex128, device=DEV)  # device buffers are refused
    code = api.lib().subapsnap_solve_batch_host(sv.ctx, params.ctypes.data, m, api.SAS_OUT_QOI,
                                                dev.data_ptr(), None, None, None)
    assert code == api.SAS_EINVAL
    sv.close()

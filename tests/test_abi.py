"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

These run without a GPU: only loading, symbol lookup and argument checks that
return before any device work.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(subapsnap_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_04825_gb300 import _build, api
    if not os.path.exists(api.LIB_PATH):
        _build.build()
    return api.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("subapsnap_setup_affine", "subapsnap_solve_batch", "subapsnap_residual"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_mirrors_the_header():
    from paper_2510_04825_gb300 import api
    for name in declared_functions():
        assert name in api.EXPORTED, name


def test_argument_checks_without_device(lib):
    from paper_2510_04825_gb300 import api
    ctx = ctypes.c_void_p()
    assert lib.subapsnap_setup_affine(None, ctypes.byref(ctx)) == api.SAS_EINVAL
    assert b"NULL" in lib.subapsnap_last_error()
    d = api.AffineDesc()
    d.n, d.r, d.s, d.K = 100, 10, 5, 2
    assert lib.subapsnap_setup_affine(ctypes.byref(d), ctypes.byref(ctx)) == api.SAS_EINVAL
    assert b"r <= s" in lib.subapsnap_last_error()
    assert lib.subapsnap_solve_batch(None, None, 0, 0, None, None, None, None) == api.SAS_EINVAL
    assert api.subapsnap_version().startswith("subapsnap")
    # the host-buffer, offline-stage and selection-variant entry points check before any device work
    assert lib.subapsnap_solve_batch_host(None, None, 4, 0, None, None, None, None) == api.SAS_EINVAL
    x = np.zeros(8)
    assert lib.subapsnap_krylov_affine(None, x.ctypes.data, 1, None, 0, 1e-8, 10, None, None) == api.SAS_EINVAL
    assert lib.subapsnap_krylov_affine(ctypes.byref(d), x.ctypes.data, 0, x.ctypes.data, 0, 1e-8, 10,
                                       None, None) == api.SAS_EINVAL
    assert b"B" in lib.subapsnap_last_error()
    assert lib.subapsnap_tsqr(None, 10, 2, 10, 0, None, 10, None) == api.SAS_EINVAL
    assert lib.subapsnap_tsqr(x.ctypes.data, 1, 2, 1, 0, x.ctypes.data, 1, None) == api.SAS_EINVAL
    cnt = ctypes.c_int32()
    assert lib.subapsnap_select_rows_union_affine(None, None, 1, 1, None, ctypes.byref(cnt)) == api.SAS_EINVAL
    assert lib.subapsnap_nearest_points(x.ctypes.data, 2, 0, x.ctypes.data, 1, x.ctypes.data) == api.SAS_EINVAL
    # entry points of the kernel-ridge snapshots, the point shards and the surrogate
    assert lib.subapsnap_krr_snapshots(None, None, 1, None, 1, 1e-8, 10, None, 1, None, None,
                                       None) == api.SAS_EINVAL
    assert lib.subapsnap_setup_kernel_shard(None, ctypes.byref(ctx)) == api.SAS_EINVAL
    assert lib.subapsnap_kernel_rows(None, None, 1, None, None) == api.SAS_EINVAL
    assert lib.subapsnap_solve_batch_rows(None, None, 1, None, None, None, None, None) == api.SAS_EINVAL
    assert lib.subapsnap_surrogate_set_anchors(None, None, None, 0) == api.SAS_EINVAL
    assert lib.subapsnap_surrogate_reset(None) == api.SAS_EINVAL
    assert lib.subapsnap_set_option(None, api.SAS_OPT_SURROGATE_F32_OUT, 1.0) == api.SAS_EINVAL


def test_product_path_has_no_oracle_import():
    """The library package must not import the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2510_04825_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True):
        src = open(path).read()
        assert "import oracle" not in src and "from oracle" not in src, path


def test_host_leverage_sampler_matches_the_oracle(lib):
    """The library's host-side leverage sampler (no GPU involved) draws the rows and
    weights the oracle draws from the same scores and uniforms, bit for bit."""
    from oracle import leverage
    from paper_2510_04825_gb300 import api
    rng = np.random.default_rng(9)
    for n, s in ((50, 20), (1000, 300), (7, 40)):
        scores = rng.uniform(0.0, 1.0, n) ** 3
        u = rng.uniform(size=s)
        J, w = api.subapsnap_sample_rows_leverage(scores, s, u)
        Jo, wo = leverage.sample_rows(scores, s, u)
        np.testing.assert_array_equal(J, Jo)
        np.testing.assert_array_equal(w, wo)
    with pytest.raises(api.SasError):
        api.subapsnap_sample_rows_leverage(np.zeros(5), 3, [0.1, 0.2, 0.3])
    with pytest.raises(api.SasError):
        api.subapsnap_sample_rows_leverage(np.ones(5), 2, [0.1, 1.0])


def test_host_nearest_points_matches_the_oracle(lib):
    from oracle import selection
    from paper_2510_04825_gb300 import api

    rng = np.random.default_rng(3)
    for m, dp, t in ((200, 1, 5), (500, 4, 7), (0, 2, 3)):
        pts = rng.uniform(size=(t, dp))
        P = rng.uniform(size=(m, dp))
        if m:
            P[:t] = pts  # exact hits
        np.testing.assert_array_equal(api.subapsnap_nearest_points(P.reshape(m, dp), pts),
                                      selection.nearest_points(P.reshape(m, dp), pts))
    # ties go to the lowest index on both sides
    pts = np.array([[0.0], [2.0], [1.0], [1.0]])
    P = np.array([[1.5], [0.5], [1.0]])
    np.testing.assert_array_equal(api.subapsnap_nearest_points(P, pts), [1, 0, 2])
    np.testing.assert_array_equal(selection.nearest_points(P, pts), [1, 0, 2])


def _affine_desc(**fields):
    from paper_2510_04825_gb300 import api
    d = api.AffineDesc()
    d.n, d.r, d.s, d.K, d.ldS = 100, 10, 20, 2, 100
    d.dtype, d.theta_rule, d.mode = api.SAS_REAL64, api.SAS_THETA_LINEAR, api.SAS_MODE_PLAIN
    for k, v in fields.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("fields,msg", [
    ({"n": 0}, b"n must be positive"),
    ({"r": 0}, b"r must be in [1, 128]"),
    ({"r": 129, "s": 200, "n": 300, "ldS": 300}, b"r must be in [1, 128]"),
    ({"s": 9}, b"need r <= s"),
    ({"s": 513, "n": 600, "ldS": 600}, b"need r <= s"),
    ({"s": 101}, b"need r <= s"),  # s > n
    ({"K": 0}, b"K must be in [1, 8]"),
    ({"K": 9}, b"K must be in [1, 8]"),
    ({"dtype": 7}, b"bad dtype"),
    ({"theta_rule": 1}, b"pencil rule needs complex128 and K = 2"),  # real dtype
    ({"theta_rule": 1, "dtype": 1, "K": 3}, b"pencil rule needs complex128 and K = 2"),
    ({"theta_rule": 2, "dtype": 1, "K": 2}, b"delay rule needs complex128 and K = 3"),
    ({"theta_rule": 9}, b"bad theta rule"),
    ({"mode": 5}, b"bad mode"),
    ({"ldS": 99}, b"ldS < n"),
    ({}, b"S must be a device pointer"),  # every field valid, S NULL
], ids=lambda v: v.decode() if isinstance(v, bytes) else None)
def test_affine_descriptor_checks(lib, fields, msg):
    """Each invalid field of the affine descriptor is refused with SAS_EINVAL and its
    message before any device work, and the context stays NULL."""
    from paper_2510_04825_gb300 import api
    d = _affine_desc(**fields)
    ctx = ctypes.c_void_p(1)
    assert lib.subapsnap_setup_affine(ctypes.byref(d), ctypes.byref(ctx)) == api.SAS_EINVAL
    assert msg in lib.subapsnap_last_error(), lib.subapsnap_last_error()
    assert ctx.value is None


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_affine_row_weights_must_be_positive_and_finite(lib, bad):
    """Row weights (leverage sampling, Sec. 4.3.3) are checked on the host before the
    device pointers."""
    from paper_2510_04825_gb300 import api
    w = np.ones(20)
    w[7] = bad
    d = _affine_desc()
    d.w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ctx = ctypes.c_void_p(1)
    assert lib.subapsnap_setup_affine(ctypes.byref(d), ctypes.byref(ctx)) == api.SAS_EINVAL
    assert b"row weights must be positive and finite" in lib.subapsnap_last_error()
    assert ctx.value is None


@pytest.mark.parametrize("fields,msg", [
    ({"n": 0}, b"n must be positive"),
    ({"d": 0}, b"d must be in [1, 16]"),
    ({"d": 17}, b"d must be in [1, 16]"),
    ({"r": 0}, b"r must be in [1, 128]"),
    ({"s": 9}, b"need r <= s"),
    ({"s": 101}, b"need r <= s"),  # s > n
    ({"mode": 5}, b"bad mode"),
    ({"ldS": 99}, b"ldS < n"),
    ({}, b"X and S must be device pointers"),
], ids=lambda v: v.decode() if isinstance(v, bytes) else None)
def test_kernel_descriptor_checks(lib, fields, msg):
    """The Gaussian-kernel descriptor's fields, as for the affine one."""
    from paper_2510_04825_gb300 import api
    d = api.KernelDesc()
    d.n, d.d, d.r, d.s, d.ldS, d.mode = 100, 8, 10, 20, 100, api.SAS_MODE_PLAIN
    for k, v in fields.items():
        setattr(d, k, v)
    ctx = ctypes.c_void_p(1)
    assert lib.subapsnap_setup_kernel(ctypes.byref(d), ctypes.byref(ctx)) == api.SAS_EINVAL
    assert msg in lib.subapsnap_last_error(), lib.subapsnap_last_error()
    assert ctx.value is None
    # a shard context skips the s <= n check (its n is the shard's points), not the others
    if fields and "s" not in fields and "n" not in fields:
        sd = api.KernelShardDesc()
        sd.base = d
        ctx2 = ctypes.c_void_p(1)
        assert lib.subapsnap_setup_kernel_shard(ctypes.byref(sd), ctypes.byref(ctx2)) == api.SAS_EINVAL
        assert msg in lib.subapsnap_last_error()
        assert ctx2.value is None

"""ctypes binding of libsubapsnap.so (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but check and convert arguments: tensors become device pointers,
the current torch stream becomes the cudaStream_t, status codes become
exceptions.  All arithmetic of the online stage runs in the library's CUDA
kernels.  Importing this module never falls back to anything: if the shared
library is missing the first call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsubapsnap.so")

SAS_OK, SAS_EINVAL, SAS_ENOMEM, SAS_ECUDA, SAS_ERANK, SAS_ETIMEOUT, SAS_ENOTSUP, SAS_ENOCONV = range(8)
SAS_FLAG_ILLCOND, SAS_FLAG_NONFINITE, SAS_FLAG_REFINE_STALL = 1, 2, 4
SAS_REAL64, SAS_COMPLEX128 = 0, 1
SAS_THETA_LINEAR, SAS_THETA_PENCIL, SAS_THETA_DELAY = 0, 1, 2
SAS_QOI_NONE, SAS_QOI_TRANSPOSE, SAS_QOI_MEAN = 0, 1, 2
SAS_MODE_PLAIN, SAS_MODE_MIXED = 0, 1
SAS_OUT_Y, SAS_OUT_XHAT, SAS_OUT_QOI = 0, 1, 3
SAS_MAX_TERMS = 8

EXPORTED = [
    "subapsnap_setup_affine", "subapsnap_setup_kernel", "subapsnap_solve_batch",
    "subapsnap_residual", "subapsnap_true_residual", "subapsnap_select_rows_affine",
    "subapsnap_destroy", "subapsnap_last_error", "subapsnap_device_status", "subapsnap_version",
    "subapsnap_set_tracing", "subapsnap_trace_read", "subapsnap_solve_batch_xhat_noalloc",
    "subapsnap_set_option", "subapsnap_reconstruct", "subapsnap_select_rows_kernel",
    "subapsnap_autotune", "subapsnap_surrogate_train", "subapsnap_surrogate_predict",
    "subapsnap_solve_batch_surrogate", "subapsnap_surrogate_weights", "subapsnap_surrogate_grad",
    "subapsnap_multi_plan_create", "subapsnap_multi_plan_launch", "subapsnap_multi_plan_destroy",
    "subapsnap_selftest_wait", "subapsnap_leverage_scores_affine", "subapsnap_sample_rows_leverage",
    "subapsnap_select_rows_union_affine", "subapsnap_nearest_points", "subapsnap_krylov_affine",
    "subapsnap_tsqr", "subapsnap_solve_batch_host", "subapsnap_krylov_affine_ex",
    "subapsnap_output_row_bytes", "subapsnap_surrogate_set_anchors", "subapsnap_surrogate_reset",
    "subapsnap_krr_snapshots", "subapsnap_setup_kernel_shard", "subapsnap_kernel_rows",
    "subapsnap_solve_batch_rows",
]
SAS_FLAG_SURROGATE, SAS_FLAG_FALLBACK = 8, 16
SAS_KERNEL_SURROGATE = 4
SAS_OPT_RECON_KERNEL, SAS_OPT_MAX_REFINE, SAS_OPT_REFINE_TOL, SAS_OPT_LS_VARIANT = 0, 1, 2, 3
SAS_OPT_ASSEMBLY_KERNEL, SAS_OPT_ASSEMBLY_SEGMENT, SAS_OPT_RECON_STORE = 4, 5, 6
SAS_OPT_HOST_CHUNK, SAS_OPT_XHAT_F32, SAS_OPT_SURROGATE_F32_OUT = 7, 8, 9
SAS_MAX_VARIANTS = 32
SAS_KRYLOV_WARM, SAS_KRYLOV_MIXED, SAS_KRYLOV_BICGSTAB = 1, 2, 4
SAS_PRECOND_JACOBI, SAS_PRECOND_POISSON = 0, 1
SAS_NOALLOC_MAX_Y = 65536
SAS_KERNEL_LS, SAS_KERNEL_RECONSTRUCT, SAS_KERNEL_RESIDUAL, SAS_KERNEL_ASSEMBLE = 0, 1, 2, 3


class SasError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"subapsnap error {code}: {msg}")
        self.code = code


class KrylovPrecond(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("ndim", ctypes.c_int32), ("dims", ctypes.c_int64 * 3),
                ("coef", ctypes.c_void_p)]


class AffineDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("r", ctypes.c_int32), ("s", ctypes.c_int32),
        ("K", ctypes.c_int32), ("dtype", ctypes.c_int32), ("theta_rule", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("S", ctypes.c_void_p), ("ldS", ctypes.c_int64),
        ("J", ctypes.POINTER(ctypes.c_int64)), ("b", ctypes.c_void_p),
        ("rowptr", ctypes.c_void_p * SAS_MAX_TERMS), ("colind", ctypes.c_void_p * SAS_MAX_TERMS),
        ("values", ctypes.c_void_p * SAS_MAX_TERMS), ("qoi_kind", ctypes.c_int32),
        ("c", ctypes.c_void_p), ("w", ctypes.POINTER(ctypes.c_double)),
    ]


class KernelDesc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("r", ctypes.c_int32), ("s", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("X", ctypes.c_void_p), ("S", ctypes.c_void_p),
        ("ldS", ctypes.c_int64), ("J", ctypes.POINTER(ctypes.c_int64)), ("b", ctypes.c_void_p),
    ]


class KernelShardDesc(ctypes.Structure):
    _fields_ = [("base", KernelDesc), ("XJ", ctypes.c_void_p), ("SJ", ctypes.c_void_p),
                ("bJ", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.subapsnap_setup_affine.argtypes = [ctypes.POINTER(AffineDesc), ctypes.POINTER(vp)]
        L.subapsnap_setup_kernel.argtypes = [ctypes.POINTER(KernelDesc), ctypes.POINTER(vp)]
        L.subapsnap_setup_kernel_shard.argtypes = [ctypes.POINTER(KernelShardDesc), ctypes.POINTER(vp)]
        L.subapsnap_kernel_rows.argtypes = [vp, vp, i64, vp, vp]
        L.subapsnap_solve_batch_rows.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp]
        L.subapsnap_solve_batch.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
        L.subapsnap_residual.argtypes = [vp, vp, i64, vp, vp, vp]
        L.subapsnap_true_residual.argtypes = [vp, vp, i64, vp, vp, vp]
        L.subapsnap_select_rows_affine.argtypes = [ctypes.POINTER(AffineDesc),
                                                   ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.POINTER(ctypes.c_double)]
        L.subapsnap_destroy.argtypes = [vp]
        L.subapsnap_destroy.restype = None
        L.subapsnap_last_error.restype = ctypes.c_char_p
        L.subapsnap_version.restype = ctypes.c_char_p
        L.subapsnap_device_status.argtypes = [vp, vp]
        L.subapsnap_set_tracing.argtypes = [vp, i32]
        L.subapsnap_set_option.argtypes = [vp, i32, ctypes.c_double]
        L.subapsnap_reconstruct.argtypes = [vp, vp, i64, vp, vp]
        L.subapsnap_output_row_bytes.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64)]
        dp_, fp_, i64p = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int64)
        L.subapsnap_surrogate_train.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_double,
                                                ctypes.c_uint64, dp_, vp]
        L.subapsnap_surrogate_predict.argtypes = [vp, vp, i64, vp, vp]
        L.subapsnap_solve_batch_surrogate.argtypes = [vp, vp, i64, i32, vp, vp, vp, ctypes.c_double,
                                                      i64p, vp]
        L.subapsnap_surrogate_weights.argtypes = [vp, i32, fp_, dp_, i64p]
        L.subapsnap_surrogate_grad.argtypes = [vp, vp, vp, i64, dp_, fp_]
        L.subapsnap_surrogate_set_anchors.argtypes = [vp, vp, vp, i64]
        L.subapsnap_surrogate_reset.argtypes = [vp]
        L.subapsnap_krr_snapshots.argtypes = [ctypes.POINTER(KernelDesc), dp_, i32, dp_, i32, ctypes.c_double,
                                              i32, vp, i64, ctypes.POINTER(ctypes.c_int32), dp_, vp]
        L.subapsnap_multi_plan_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), i64p,
                                                  i32, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                  ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.subapsnap_multi_plan_launch.argtypes = [vp, i32, vp]
        L.subapsnap_multi_plan_destroy.argtypes = [vp]
        L.subapsnap_multi_plan_destroy.restype = None
        L.subapsnap_selftest_wait.argtypes = [vp, ctypes.c_double, vp]
        L.subapsnap_autotune.argtypes = [vp, vp, i64, i32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int32), vp]
        L.subapsnap_select_rows_kernel.argtypes = [ctypes.POINTER(KernelDesc),
                                                   ctypes.POINTER(ctypes.c_double),
                                                   ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.POINTER(ctypes.c_double)]
        L.subapsnap_solve_batch_xhat_noalloc.argtypes = [vp, vp, i64, vp, vp, vp, vp]
        L.subapsnap_trace_read.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int64)]
        L.subapsnap_leverage_scores_affine.argtypes = [ctypes.POINTER(AffineDesc), vp, vp]
        L.subapsnap_sample_rows_leverage.argtypes = [vp, i64, i32, vp, vp, vp, ctypes.POINTER(ctypes.c_int32)]
        L.subapsnap_select_rows_union_affine.argtypes = [ctypes.POINTER(AffineDesc), vp, i32, i32, vp,
                                                         ctypes.POINTER(ctypes.c_int32)]
        L.subapsnap_nearest_points.argtypes = [vp, i64, i32, vp, i32, vp]
        L.subapsnap_krylov_affine.argtypes = [ctypes.POINTER(AffineDesc), vp, i32, vp, i32, ctypes.c_double,
                                              i32, vp, vp]
        L.subapsnap_tsqr.argtypes = [vp, i64, i32, i64, i32, vp, i64, vp]
        L.subapsnap_solve_batch_host.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp]
        L.subapsnap_krylov_affine_ex.argtypes = [ctypes.POINTER(AffineDesc), vp, i32, vp, i32, ctypes.c_double,
                                                 i32, ctypes.POINTER(KrylovPrecond), vp, vp]
        for name in ("subapsnap_setup_affine", "subapsnap_setup_kernel", "subapsnap_solve_batch",
                     "subapsnap_residual", "subapsnap_true_residual", "subapsnap_select_rows_affine",
                     "subapsnap_device_status", "subapsnap_set_tracing", "subapsnap_trace_read",
                     "subapsnap_solve_batch_xhat_noalloc", "subapsnap_set_option",
                     "subapsnap_reconstruct", "subapsnap_select_rows_kernel",
                     "subapsnap_autotune", "subapsnap_surrogate_train",
                     "subapsnap_surrogate_predict", "subapsnap_solve_batch_surrogate",
                     "subapsnap_surrogate_weights", "subapsnap_surrogate_grad",
                     "subapsnap_multi_plan_create", "subapsnap_multi_plan_launch",
                     "subapsnap_selftest_wait", "subapsnap_leverage_scores_affine",
                     "subapsnap_sample_rows_leverage", "subapsnap_select_rows_union_affine",
                     "subapsnap_nearest_points", "subapsnap_krylov_affine", "subapsnap_tsqr",
                     "subapsnap_solve_batch_host", "subapsnap_krylov_affine_ex",
                     "subapsnap_surrogate_set_anchors", "subapsnap_surrogate_reset",
                     "subapsnap_krr_snapshots", "subapsnap_setup_kernel_shard",
                     "subapsnap_kernel_rows", "subapsnap_solve_batch_rows"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(code: int):
    if code != SAS_OK:
        raise SasError(code, lib().subapsnap_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _affine_desc(n, r, s, blocks, S, J, b, theta_rule, mode, qoi_kind=SAS_QOI_NONE, c=None,
                 complex_valued=False, w=None):
    """Fill the C descriptor.  ``blocks`` is a list of (rowptr int64, colind int32,
    values float64) CUDA tensors; S is (r, n) row-major in memory, i.e. the
    column-major n x r matrix with ldS = n."""
    d = AffineDesc()
    d.n, d.r, d.s, d.K = int(n), int(r), int(s), len(blocks)
    d.dtype = SAS_COMPLEX128 if complex_valued else SAS_REAL64
    d.theta_rule, d.mode = theta_rule, mode
    d.S, d.ldS = _ptr(S), int(n)
    if J is not None:
        Jh = np.ascontiguousarray(np.asarray(J, dtype=np.int64))
        d.J = Jh.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d._J_keep = Jh
    d.b = _ptr(b) if b is not None else None
    for k, (rp, ci, va) in enumerate(blocks):
        d.rowptr[k], d.colind[k], d.values[k] = _ptr(rp), _ptr(ci), _ptr(va)
    d.qoi_kind = qoi_kind
    d.c = _ptr(c) if c is not None else None
    if w is not None:
        wh = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        d.w = wh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d._w_keep = wh
    return d


def subapsnap_version() -> str:
    return lib().subapsnap_version().decode()


def subapsnap_setup_affine(desc: AffineDesc) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().subapsnap_setup_affine(ctypes.byref(desc), ctypes.byref(ctx)))
    return ctx


def _kernel_desc(n, d, r, s, X, S, J, b, mode):
    """Fill the C descriptor of the Gaussian-kernel family.  X is (N, d) row-major,
    S is (r, N) row-major in memory (column-major N x r, ldS = N)."""
    k = KernelDesc()
    k.n, k.d, k.r, k.s, k.mode = int(n), int(d), int(r), int(s), mode
    k.X, k.S, k.ldS = _ptr(X), _ptr(S), int(n)
    Jh = np.ascontiguousarray(np.asarray(J, dtype=np.int64))
    k.J = Jh.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    k._J_keep = Jh
    k.b = _ptr(b)
    return k


def subapsnap_setup_kernel(desc: KernelDesc) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().subapsnap_setup_kernel(ctypes.byref(desc), ctypes.byref(ctx)))
    return ctx


def subapsnap_setup_kernel_shard(desc: KernelShardDesc) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().subapsnap_setup_kernel_shard(ctypes.byref(desc), ctypes.byref(ctx)))
    return ctx


def subapsnap_kernel_rows(ctx, params, m: int, M, stream=None):
    """M (device, m x s x r doubles; each parameter's block column-major) = the context's rows."""
    _check(lib().subapsnap_kernel_rows(ctx, _ptr(params), int(m), _ptr(M), _stream(stream)))


def subapsnap_solve_batch_rows(ctx, params, m: int, M, Y, flags=None, rho=None, stream=None):
    _check(lib().subapsnap_solve_batch_rows(ctx, _ptr(params), int(m), _ptr(M), _ptr(Y), _ptr(flags),
                                            _ptr(rho), _stream(stream)))


def subapsnap_select_rows_affine(desc: AffineDesc, p_sel, s: int):
    ps = np.ascontiguousarray(np.atleast_1d(np.asarray(p_sel, dtype=np.float64)))
    J = np.zeros(s, dtype=np.int64)
    gaps = np.zeros(s, dtype=np.float64)
    _check(lib().subapsnap_select_rows_affine(
        ctypes.byref(desc), ps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        J.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        gaps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return J, gaps


def subapsnap_select_rows_kernel(desc: KernelDesc, p_sel, s: int):
    ps = np.ascontiguousarray(np.asarray(p_sel, dtype=np.float64).reshape(2))
    J = np.zeros(s, dtype=np.int64)
    gaps = np.zeros(s, dtype=np.float64)
    _check(lib().subapsnap_select_rows_kernel(
        ctypes.byref(desc), ps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        J.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        gaps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return J, gaps


def subapsnap_output_row_bytes(ctx, out_kind: int) -> int:
    b = ctypes.c_int64()
    _check(lib().subapsnap_output_row_bytes(ctx, int(out_kind), ctypes.byref(b)))
    return b.value


def _check_out(ctx, out_kind, out, m):
    """The output buffer must hold m rows of what the context writes for out_kind;
    a 2-D buffer's rows must be exactly one parameter's output (so that a float32
    x_hat buffer is never handed to a context that writes float64)."""
    row = subapsnap_output_row_bytes(ctx, out_kind)
    if hasattr(out, "element_size"):
        esize, shape = out.element_size(), tuple(out.shape)
    else:
        arr = np.asarray(out)
        esize, shape = arr.itemsize, arr.shape
    nbytes = esize * int(np.prod(shape)) if shape else esize
    if nbytes < int(m) * row:
        raise ValueError(f"output buffer holds {nbytes} bytes; {int(m)} rows need {int(m) * row}")
    if len(shape) == 2 and shape[1] * esize != row:
        raise ValueError(f"output rows are {shape[1] * esize} bytes; the context writes {row} per row")


def subapsnap_solve_batch(ctx, params, m: int, out_kind: int, out, flags=None, rho=None,
                          stream=None):
    _check_out(ctx, out_kind, out, m)
    _check(lib().subapsnap_solve_batch(ctx, _ptr(params), int(m), int(out_kind), _ptr(out),
                                       _ptr(flags), _ptr(rho), _stream(stream)))


def subapsnap_solve_batch_xhat_noalloc(ctx, params, m: int, out, flags=None, rho=None,
                                       stream=None):
    _check(lib().subapsnap_solve_batch_xhat_noalloc(ctx, _ptr(params), int(m), _ptr(out),
                                                    _ptr(flags), _ptr(rho), _stream(stream)))


def subapsnap_autotune(ctx, params, m: int, reps: int = 3, stream=None):
    """Time every least-squares launch shape; returns (chosen index, times in ms)."""
    times = (ctypes.c_double * SAS_MAX_VARIANTS)()
    chosen = ctypes.c_int32()
    _check(lib().subapsnap_autotune(ctx, _ptr(params), int(m), int(reps), times,
                                    ctypes.byref(chosen), _stream(stream)))
    return chosen.value, [t for t in times]


def subapsnap_leverage_scores_affine(desc: AffineDesc, p_sel) -> np.ndarray:
    """Leverage scores of [A(p_sel) S, b] (host array of n doubles)."""
    sc = np.empty(desc.n, dtype=np.float64)
    ps = np.ascontiguousarray(np.atleast_1d(np.asarray(p_sel, dtype=np.float64)))
    _check(lib().subapsnap_leverage_scores_affine(ctypes.byref(desc), ps.ctypes.data_as(ctypes.c_void_p),
                                                  sc.ctypes.data_as(ctypes.c_void_p)))
    return sc


def subapsnap_sample_rows_leverage(scores, s: int, u):
    """(J, w): s inverse-CDF draws on the uniforms u, duplicates merged into weights."""
    sc = np.ascontiguousarray(np.asarray(scores, dtype=np.float64))
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    J = np.empty(int(s), dtype=np.int64)
    w = np.empty(int(s), dtype=np.float64)
    cnt = ctypes.c_int32()
    _check(lib().subapsnap_sample_rows_leverage(sc.ctypes.data_as(ctypes.c_void_p), int(sc.size), int(s),
                                                uu.ctypes.data_as(ctypes.c_void_p),
                                                J.ctypes.data_as(ctypes.c_void_p),
                                                w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
    return J[:cnt.value].copy(), w[:cnt.value].copy()


def subapsnap_select_rows_union_affine(desc: AffineDesc, points, s_each: int) -> np.ndarray:
    """Union of the CPQR picks at each row of ``points`` (t x dp), first appearance order."""
    pts = np.ascontiguousarray(np.atleast_2d(np.asarray(points, dtype=np.float64)))
    t = pts.shape[0]
    J = np.empty(t * int(s_each), dtype=np.int64)
    cnt = ctypes.c_int32()
    _check(lib().subapsnap_select_rows_union_affine(ctypes.byref(desc), pts.ctypes.data_as(ctypes.c_void_p),
                                                    int(t), int(s_each), J.ctypes.data_as(ctypes.c_void_p),
                                                    ctypes.byref(cnt)))
    return J[:cnt.value].copy()


def subapsnap_nearest_points(params, points) -> np.ndarray:
    """Index of the nearest row of ``points`` for every row of ``params``."""
    P = np.ascontiguousarray(np.atleast_2d(np.asarray(params, dtype=np.float64)))
    pts = np.ascontiguousarray(np.atleast_2d(np.asarray(points, dtype=np.float64)))
    idx = np.empty(P.shape[0], dtype=np.int32)
    _check(lib().subapsnap_nearest_points(P.ctypes.data_as(ctypes.c_void_p), int(P.shape[0]), int(P.shape[1]),
                                          pts.ctypes.data_as(ctypes.c_void_p), int(pts.shape[0]),
                                          idx.ctypes.data_as(ctypes.c_void_p)))
    return idx


def subapsnap_krylov_affine(desc: AffineDesc, params, X, warm: bool = False, tol: float = 1e-12,
                            maxit: int = 20000, allow_noconv: bool = False, mixed: bool = False,
                            precond=None, method: str = "cg"):
    """Batched snapshot solves A(p_j) x_j = b.  X: CUDA tensor (B, n), row j = x_j
    (the column-major n x B matrix).  precond: None (Jacobi) or a dict with keys
    "dims" (grid sizes) and "coef" (B x 4: alpha re/im, beta re/im) for the fast
    Poisson preconditioner.  Returns (iterations, true relative residuals)."""
    flags = (SAS_KRYLOV_WARM if warm else 0) | (SAS_KRYLOV_MIXED if mixed else 0)
    if method == "bicgstab":
        flags |= SAS_KRYLOV_BICGSTAB
    elif method != "cg":
        raise ValueError("method must be 'cg' or 'bicgstab'")
    P = np.ascontiguousarray(np.atleast_2d(np.asarray(params, dtype=np.float64)))
    B = int(X.shape[0])
    it = np.zeros(B, dtype=np.int32)
    rel = np.zeros(B, dtype=np.float64)
    pc = None
    if precond is not None:
        coef = np.ascontiguousarray(np.asarray(precond["coef"], dtype=np.float64).reshape(B, 4))
        dims = list(precond["dims"])
        pc = KrylovPrecond()
        pc.kind, pc.ndim = SAS_PRECOND_POISSON, len(dims)
        for a, v in enumerate(dims):
            pc.dims[a] = int(v)
        pc.coef = coef.ctypes.data
        pc._coef_keep = coef
    code = lib().subapsnap_krylov_affine_ex(ctypes.byref(desc), P.ctypes.data_as(ctypes.c_void_p), B, _ptr(X),
                                            flags, float(tol), int(maxit),
                                            ctypes.byref(pc) if pc is not None else None,
                                            it.ctypes.data_as(ctypes.c_void_p), rel.ctypes.data_as(ctypes.c_void_p))
    if not (allow_noconv and code == SAS_ENOCONV):
        _check(code)
    return it, rel


def subapsnap_krr_snapshots(X, b, sigma, lam, Xout, tol: float = 1e-10, maxit: int = 10000, stream=None):
    """Kernel-ridge snapshots by multishift CG: X (N, d) and b (N,) float64 CUDA tensors, sigma and
    lam host sequences; Xout a float64 CUDA tensor of shape (len(sigma) * len(lam), N) whose row
    a * len(lam) + b receives the solution for (sigma[a], lam[b]).  Returns (iterations, true
    relative residuals) as numpy arrays."""
    import torch
    N, d = int(X.shape[0]), int(X.shape[1])
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    lm = np.ascontiguousarray(lam, dtype=np.float64)
    nc = len(sig) * len(lm)
    if tuple(Xout.shape) != (nc, N) or Xout.dtype != torch.float64 or not Xout.is_contiguous():
        raise ValueError(f"Xout must be a contiguous float64 tensor of shape ({nc}, {N})")
    desc = KernelDesc(n=N, d=d, r=0, s=0, mode=0, X=_ptr(X), S=None, ldS=0, J=None, b=_ptr(b))
    its = np.zeros(nc, dtype=np.int32)
    res = np.zeros(nc, dtype=np.float64)
    _check(lib().subapsnap_krr_snapshots(
        ctypes.byref(desc), sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(sig),
        lm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(lm), float(tol), int(maxit), _ptr(Xout), N,
        its.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        _stream(stream)))
    return its, res


def subapsnap_tsqr(X, Q=None, complex_valued: bool | None = None) -> np.ndarray:
    """Thin QR of the column-major n x r matrix held by the CUDA tensor X of shape (r, n).
    Q (same shape, may be X) receives the orthonormal factor; returns R (r x r, host)."""
    r, n = int(X.shape[0]), int(X.shape[1])
    cplx = X.is_complex() if complex_valued is None else complex_valued
    Q = X if Q is None else Q
    R = np.zeros((r, r), dtype=np.complex128 if cplx else np.float64)  # R[j, i] = R_ij (column-major)
    _check(lib().subapsnap_tsqr(_ptr(X), n, r, n, SAS_COMPLEX128 if cplx else SAS_REAL64, _ptr(Q), n,
                                R.ctypes.data_as(ctypes.c_void_p)))
    return np.ascontiguousarray(R.T)


def _hptr(a):
    """Host pointer of a CPU tensor or a numpy array (None passes through)."""
    if a is None:
        return None
    if hasattr(a, "is_cuda"):
        if a.is_cuda:
            raise ValueError("expected a host (CPU) tensor")
        if not a.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous array")
    return a.ctypes.data


def subapsnap_solve_batch_host(ctx, params, m: int, out_kind: int, out, flags=None, rho=None, stream=None):
    """solve_batch with host buffers (CPU tensors or numpy arrays); returns when out is filled."""
    _check_out(ctx, out_kind, out, m)
    _check(lib().subapsnap_solve_batch_host(ctx, _hptr(params), int(m), int(out_kind), _hptr(out),
                                            _hptr(flags), _hptr(rho), _stream(stream)))


def subapsnap_reconstruct(ctx, Y, m: int, out, stream=None):
    _check_out(ctx, SAS_OUT_XHAT, out, m)
    _check(lib().subapsnap_reconstruct(ctx, _ptr(Y), int(m), _ptr(out), _stream(stream)))


def subapsnap_residual(ctx, params, m: int, Y, rho, stream=None):
    _check(lib().subapsnap_residual(ctx, _ptr(params), int(m), _ptr(Y), _ptr(rho), _stream(stream)))


def subapsnap_true_residual(ctx, params, m: int, X, rho, stream=None):
    _check(lib().subapsnap_true_residual(ctx, _ptr(params), int(m), _ptr(X), _ptr(rho),
                                         _stream(stream)))


def subapsnap_device_status(ctx, stream=None) -> int:
    return int(lib().subapsnap_device_status(ctx, _stream(stream)))


def subapsnap_set_option(ctx, key: int, value: float):
    _check(lib().subapsnap_set_option(ctx, int(key), float(value)))


def subapsnap_set_tracing(ctx, enable: bool):
    _check(lib().subapsnap_set_tracing(ctx, 1 if enable else 0))


def subapsnap_trace_read(ctx, kernel_class: int):
    """(total milliseconds, launches) of one kernel class since the last read."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(lib().subapsnap_trace_read(ctx, kernel_class, ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def subapsnap_surrogate_train(ctx, P, Y, epochs: int, batch: int, lr: float, seed: int = 0,
                              stream=None):
    """Train the network on (P, Y) device tensors; returns the mean loss of every epoch."""
    losses = np.zeros(max(epochs, 1), dtype=np.float64)
    _check(lib().subapsnap_surrogate_train(ctx, _ptr(P), _ptr(Y), int(P.shape[0]), int(epochs),
                                           int(batch), float(lr), int(seed),
                                           losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           _stream(stream)))
    return losses[:epochs]


def subapsnap_surrogate_predict(ctx, params, m: int, Yhat, stream=None):
    _check(lib().subapsnap_surrogate_predict(ctx, _ptr(params), int(m), _ptr(Yhat), _stream(stream)))


def subapsnap_solve_batch_surrogate(ctx, params, m: int, out_kind: int, out, flags=None, rho=None,
                                    gate_tol: float = 1e-6, stream=None) -> int:
    acc = ctypes.c_int64()
    _check_out(ctx, out_kind, out, m)
    _check(lib().subapsnap_solve_batch_surrogate(ctx, _ptr(params), int(m), int(out_kind), _ptr(out),
                                                 _ptr(flags), _ptr(rho), float(gate_tol),
                                                 ctypes.byref(acc), _stream(stream)))
    return acc.value


def subapsnap_surrogate_reset(ctx):
    """Discard the network; the next training starts from a fresh one."""
    _check(lib().subapsnap_surrogate_reset(ctx))


def subapsnap_surrogate_set_anchors(ctx, P=None, Y=None):
    """Anchors (device float64 P: n x dp, Y: n x r) for the next training; None clears."""
    n = 0 if P is None else int(P.shape[0])
    _check(lib().subapsnap_surrogate_set_anchors(ctx, _ptr(P) if n else None, _ptr(Y) if n else None, n))


def subapsnap_surrogate_weights(ctx, get: bool, theta=None, norm=None) -> int:
    """theta: numpy float32 (nparam), norm: numpy float64 (2 (dp + r)); returns nparam."""
    n = ctypes.c_int64()
    tp = theta.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if theta is not None else None
    npp = norm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if norm is not None else None
    _check(lib().subapsnap_surrogate_weights(ctx, 1 if get else 0, tp, npp, ctypes.byref(n)))
    return n.value


def subapsnap_surrogate_grad(ctx, X, Yn, nparam: int):
    """One forward/backward on device (X, Yn); returns (loss, gradients float32)."""
    loss = ctypes.c_double()
    g = np.zeros(nparam, dtype=np.float32)
    _check(lib().subapsnap_surrogate_grad(ctx, _ptr(X), _ptr(Yn), int(X.shape[0]), ctypes.byref(loss),
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return loss.value, g


def subapsnap_multi_plan_create(ctxs, params, out_kind: int, outs, flags=None, rho=None):
    """One persistent launch over several contexts; params/outs/flags/rho are lists of tensors."""
    n = len(ctxs)
    VP = ctypes.c_void_p * n
    arr_ctx = VP(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    arr_p = VP(*[_ptr(t) for t in params])
    arr_o = VP(*[_ptr(t) for t in outs])
    arr_f = VP(*[_ptr(t) for t in flags]) if flags is not None else None
    arr_r = VP(*[_ptr(t) for t in rho]) if rho is not None else None
    m = (ctypes.c_int64 * n)(*[int(t.shape[0]) for t in params])
    plan = ctypes.c_void_p()
    _check(lib().subapsnap_multi_plan_create(arr_ctx, n, arr_p, m, int(out_kind), arr_o, arr_f, arr_r,
                                             ctypes.byref(plan)))
    return plan


def subapsnap_multi_plan_launch(plan, use_graph: bool = False, stream=None):
    _check(lib().subapsnap_multi_plan_launch(plan, 1 if use_graph else 0, _stream(stream)))


def subapsnap_multi_plan_destroy(plan):
    lib().subapsnap_multi_plan_destroy(plan)


def subapsnap_selftest_wait(ctx, seconds: float = 0.2, stream=None) -> int:
    """Status the bounded-wait self-test records (SAS_ETIMEOUT when the mechanism works)."""
    return int(lib().subapsnap_selftest_wait(ctx, float(seconds), _stream(stream)))


def subapsnap_destroy(ctx):
    lib().subapsnap_destroy(ctx)

"""Thin Python binding of libxm (include/xm.h): argument marshalling only.

Every function keeps the C name and forwards torch CUDA tensors as device pointers; all
arithmetic happens in libxm's CUDA kernels.  There is no CPU fallback: if libxm.so is
missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxm.so")

XM_OK, XM_EINVAL, XM_EDISCONNECTED, XM_ECUDA, XM_ENOMEM, XM_ENOCONV, XM_ENUMERIC, \
    XM_ETIMEOUT, XM_ENOTCERT = range(9)
XM_FP64, XM_FP32_BULK, XM_BF16Q_BULK = 0, 1, 2
XM_STORE_FP64, XM_STORE_FP32, XM_STORE_BF16, XM_STORE_ALL, XM_STORE_FACTORED = 1, 2, 4, 7, 8
XM_MAX_RANK = 8
XM_BUILD_AUTO, XM_BUILD_FP64, XM_BUILD_SPLIT_BF16 = 0, 1, 2
STATUS_NAMES = {0: "XM_OK", 1: "XM_EINVAL", 2: "XM_EDISCONNECTED", 3: "XM_ECUDA", 4: "XM_ENOMEM",
                5: "XM_ENOCONV", 6: "XM_ENUMERIC", 7: "XM_ETIMEOUT", 8: "XM_ENOTCERT"}


class XmOpts(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_int), ("r_max", ctypes.c_int), ("prec", ctypes.c_int),
                ("grad_tol_rel", ctypes.c_double), ("bulk_tol_rel", ctypes.c_double),
                ("cert_tau_rel", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("max_tcg", ctypes.c_int), ("max_polish", ctypes.c_int),
                ("lanczos_max", ctypes.c_int), ("lanczos_tol", ctypes.c_double),
                ("time_limit_s", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("verbose", ctypes.c_int), ("init_jitter", ctypes.c_double),
                ("scale_reg", ctypes.c_double), ("precond", ctypes.c_int),
                ("bulk_stall", ctypes.c_int), ("cert_lobpcg", ctypes.c_int),
                ("bf16_hvp_until", ctypes.c_double)]


class XmInfo(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("grad_norm", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("lambda_min_deflated", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("dual", ctypes.c_double),
                ("rho_hat", ctypes.c_double), ("eta", ctypes.c_double),
                ("eta_robust", ctypes.c_double), ("rank", ctypes.c_int),
                ("certified", ctypes.c_int), ("n_sweeps", ctypes.c_int),
                ("n_sweeps_fp64", ctypes.c_int), ("n_outer", ctypes.c_int),
                ("n_tcg", ctypes.c_int), ("n_lanczos", ctypes.c_int), ("n_escapes", ctypes.c_int),
                ("t_solve_s", ctypes.c_double), ("t_cert_s", ctypes.c_double),
                ("t_build_s", ctypes.c_double), ("qy_ms_fp32", ctypes.c_double),
                ("qy_ms_fp64", ctypes.c_double), ("lanczos_converged", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class XmAdjInfo(ctypes.Structure):
    _fields_ = [("res_rel", ctypes.c_double), ("g_norm", ctypes.c_double),
                ("grad_norm_Y", ctypes.c_double), ("n_refine", ctypes.c_int),
                ("n_cg", ctypes.c_int), ("n_sweeps_fp32", ctypes.c_int),
                ("n_sweeps_fp64", ctypes.c_int), ("t_lambda_s", ctypes.c_double),
                ("t_resid_s", ctypes.c_double), ("t_total_s", ctypes.c_double),
                ("launches", ctypes.c_long), ("dense_precond", ctypes.c_int),
                ("gamma", ctypes.c_double), ("t_precond_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class XmBatchInfo(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("grad_norm", ctypes.c_double),
                ("lambda_min", ctypes.c_double), ("lambda_min_deflated", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("dual", ctypes.c_double),
                ("rho_hat", ctypes.c_double), ("eta", ctypes.c_double),
                ("eta_robust", ctypes.c_double), ("t_begin_ns", ctypes.c_ulonglong),
                ("t_end_ns", ctypes.c_ulonglong), ("t_cert_ns", ctypes.c_ulonglong),
                ("t_polish_ns", ctypes.c_ulonglong), ("N", ctypes.c_int), ("status", ctypes.c_int),
                ("rank", ctypes.c_int), ("certified", ctypes.c_int), ("n_sweeps", ctypes.c_int),
                ("n_sweeps_fp64", ctypes.c_int), ("n_outer", ctypes.c_int), ("n_tcg", ctypes.c_int),
                ("n_lanczos", ctypes.c_int), ("n_escapes", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class XmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libxm.so from the package directory (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libxm.so not found at {LIB_PATH}; run paper_2502_04640_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "xm_abi_version": (ctypes.c_int, []),
        "xm_default_opts": (None, [ctypes.POINTER(XmOpts)]),
        "xm_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
        "xm_destroy": (None, [_P]),
        "xm_last_error": (ctypes.c_char_p, []),
        "xm_sync": (ctypes.c_int, [_P]),
        "xm_selftest_wait": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_int]),
        "xm_build_Q": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P,
                                      ctypes.c_uint, ctypes.POINTER(_P)]),
        "xm_qmat_from_dense": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_uint, ctypes.POINTER(_P)]),
        "xm_qmat_to_dense": (ctypes.c_int, [_P, _P, _P]),
        "xm_qmat_dims": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_uint)]),
        "xm_free_Q": (ctypes.c_int, [_P, _P]),
        "xm_set_build_mode": (ctypes.c_int, [_P, ctypes.c_int]),
        "xm_qmat_build_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_double)]),
        "xm_qy": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P]),
        "xm_qy_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P]),
        "xm_bench_qy": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "xm_last_launch_count": (ctypes.c_long, []),
        "xm_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(XmOpts), ctypes.c_int, _P, _P, _P, _P, _P,
                                    ctypes.POINTER(XmInfo)]),
        "xm_certify": (ctypes.c_int, [_P, _P, ctypes.POINTER(XmOpts), ctypes.c_int, _P, _P, _P,
                                      ctypes.POINTER(XmInfo)]),
        "xm_pipeline_host": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P, _P, _P,
                                            _P, ctypes.POINTER(XmOpts), _P, _P, ctypes.POINTER(XmInfo)]),
        "xm_recover_tp": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P, _P,
                                         _P, _P, _P, _P]),
        "xm_solve_xm2": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P,
                                        ctypes.POINTER(XmOpts), ctypes.c_double, _P, _P, _P, _P, _P,
                                        ctypes.POINTER(XmInfo), ctypes.POINTER(XmInfo)]),
        "xm_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
        "xm_batch_free": (ctypes.c_int, [_P, _P]),
        "xm_batch_autotune": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "xm_batch_cluster": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int]),
        "xm_batch_launches": (ctypes.c_int, [_P, _P, _P, _P]),
        "xm_solve_batched": (ctypes.c_int, [_P, _P, ctypes.POINTER(XmOpts), _P, _P,
                                            ctypes.POINTER(XmBatchInfo)]),
        "xm_qfact_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P,
                                           ctypes.POINTER(_P)]),
        "xm_qy_factored": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, _P]),
        "xm_qfact_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t),
                                         ctypes.POINTER(ctypes.c_double)]),
        "xm_qfact_free": (ctypes.c_int, [_P, _P]),
        "xm_spd_inverse": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
        "xm_backward": (ctypes.c_int, [_P, _P, ctypes.POINTER(XmOpts), ctypes.c_int, _P, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P,
                                       ctypes.POINTER(XmAdjInfo)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, allow=(XM_OK,)) -> int:
    if status not in allow:
        msg = lib().xm_last_error()
        raise XmError(status, msg.decode() if msg else "")
    return status


def _ptr(t) -> int | None:
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def xm_default_opts(**overrides) -> XmOpts:
    o = XmOpts()
    lib().xm_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"xm_opts has no field {k}")
        setattr(o, k, v)
    return o


class Context:
    """An xm_ctx on one device, issuing work on the torch current stream of that device."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libxm needs a CUDA device")
        torch.cuda.set_device(device)
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.device = device
        self.stream = s
        h = _P()
        _check(lib().xm_create(ctypes.byref(h), device, _P(s.cuda_stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().xm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class QMat:
    """Owning handle of an xm_qmat."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        N, n, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_uint()
        _check(lib().xm_qmat_dims(h, ctypes.byref(N), ctypes.byref(n), ctypes.byref(m)))
        self.N, self.n, self.mask = N.value, n.value, m.value

    def free(self):
        if getattr(self, "h", None):
            lib().xm_free_Q(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def xm_build_Q(ctx: Context, N: int, M: int, cam, lmk, ukp, w, store_mask: int = XM_STORE_ALL) -> QMat:
    """cam, lmk: int32 CUDA tensors [E]; ukp: float64 [E, 3]; w: float64 [E]."""
    import torch
    E = int(cam.shape[0])
    for t, dt in ((cam, torch.int32), (lmk, torch.int32), (ukp, torch.float64), (w, torch.float64)):
        if t.dtype != dt:
            raise TypeError(f"expected {dt}, got {t.dtype}")
    h = _P()
    _check(lib().xm_build_Q(ctx.h, N, M, E, _ptr(cam), _ptr(lmk), _ptr(ukp), _ptr(w), store_mask,
                            ctypes.byref(h)))
    return QMat(ctx, h)


def xm_set_build_mode(ctx: Context, mode: int) -> None:
    """XM_BUILD_AUTO / XM_BUILD_FP64 / XM_BUILD_SPLIT_BF16 for later xm_build_Q calls."""
    _check(lib().xm_set_build_mode(ctx.h, mode))


def xm_qmat_build_info(q: QMat) -> tuple[int, float]:
    """(update path XM_BUILD_*, its device seconds) of a Q built by xm_build_Q."""
    path, t = ctypes.c_int(), ctypes.c_double()
    _check(lib().xm_qmat_build_info(q.h, ctypes.byref(path), ctypes.byref(t)))
    return path.value, t.value


def xm_qmat_from_dense(ctx: Context, Q, store_mask: int = XM_STORE_ALL) -> QMat:
    import torch
    if Q.dtype != torch.float64 or Q.dim() != 2 or Q.shape[0] != Q.shape[1] or Q.shape[0] % 3:
        raise ValueError("Q must be a square float64 CUDA tensor of size 3N")
    h = _P()
    _check(lib().xm_qmat_from_dense(ctx.h, Q.shape[0] // 3, _ptr(Q), store_mask, ctypes.byref(h)))
    return QMat(ctx, h)


def xm_qmat_to_dense(q: QMat):
    import torch
    out = torch.empty((q.n, q.n), dtype=torch.float64, device=f"cuda:{q.ctx.device}")
    _check(lib().xm_qmat_to_dense(q.ctx.h, q.h, _ptr(out)))
    return out


def xm_qy(q: QMat, Y, prec: int = XM_FP64):
    """W = Q Y for an n x r CUDA tensor Y (float64 for XM_FP64, float32 otherwise)."""
    import torch
    want = torch.float64 if prec == XM_FP64 else torch.float32
    if Y.dtype != want or Y.dim() != 2 or Y.shape[0] != q.n:
        raise ValueError(f"Y must be {want} of shape (n={q.n}, r)")
    Y = Y.contiguous()
    W = torch.empty_like(Y)
    _check(lib().xm_qy(q.ctx.h, q.h, prec, Y.shape[1], _ptr(Y), _ptr(W)))
    return W


class QFact:
    """Owning handle of an xm_qfact (the factored Q operator)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        N, M, E = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        nb, ts = ctypes.c_size_t(), ctypes.c_double()
        _check(lib().xm_qfact_info(h, ctypes.byref(N), ctypes.byref(M), ctypes.byref(E), ctypes.byref(nb),
                                   ctypes.byref(ts)))
        self.N, self.M, self.E, self.n = N.value, M.value, E.value, 3 * N.value
        self.bytes, self.t_setup_s = nb.value, ts.value

    def free(self):
        if getattr(self, "h", None):
            lib().xm_qfact_free(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def xm_qfact_create(ctx: Context, N: int, M: int, cam, lmk, ukp, w) -> QFact:
    """Factored Q operator from observation tensors (as for xm_build_Q)."""
    h = _P()
    _check(lib().xm_qfact_create(ctx.h, N, M, int(cam.shape[0]), _ptr(cam), _ptr(lmk), _ptr(ukp), _ptr(w),
                                 ctypes.byref(h)))
    return QFact(ctx, h)


def xm_qy_factored(f: QFact, Y):
    """W = Q Y by the factored operator for an n x r float64 CUDA tensor Y."""
    import torch
    if Y.dtype != torch.float64 or Y.dim() != 2 or Y.shape[0] != f.n:
        raise ValueError(f"Y must be float64 of shape (n={f.n}, r)")
    Y = Y.contiguous()
    W = torch.empty_like(Y)
    _check(lib().xm_qy_factored(f.ctx.h, f.h, Y.shape[1], _ptr(Y), _ptr(W)))
    return W


def xm_spd_inverse(ctx: Context, A):
    """In place: A <- A^{-1} for a symmetric positive definite float32 CUDA tensor A (n x n).

    Symmetric, so the row-major tensor is its own column-major layout; returns A."""
    import torch
    if A.dtype != torch.float32 or A.dim() != 2 or A.shape[0] != A.shape[1] or not A.is_contiguous():
        raise ValueError("A must be a contiguous square float32 tensor")
    n = A.shape[0]
    _check(lib().xm_spd_inverse(ctx.h, n, _ptr(A), max(n, 1)))
    return A


def xm_bench_qy(q: QMat, prec: int, r: int, iters: int = 20):
    mean, mn = ctypes.c_double(), ctypes.c_double()
    _check(lib().xm_bench_qy(q.ctx.h, q.h, prec, r, iters, ctypes.byref(mean), ctypes.byref(mn)))
    return mean.value, mn.value


def xm_selftest_wait(ctx: Context, polls: int, arrive: bool) -> int:
    """Bounded-wait self-check: XM_OK when the barrier is arrived on, XM_ETIMEOUT when not."""
    return _check(lib().xm_selftest_wait(ctx.h, polls, 1 if arrive else 0), (XM_OK, XM_ETIMEOUT))


def xm_last_launch_count() -> int:
    return int(lib().xm_last_launch_count())


def xm_solve(q: QMat, opts: XmOpts | None = None, Y0=None, allow_notcert: bool = True):
    """Returns dict(Y (n x 8 float64), R (N x 3 x 3), s (N), G (N x 3 x 3, G_i = s_i R_i),
    info (dict), status)."""
    import torch
    dev = f"cuda:{q.ctx.device}"
    opts = opts or xm_default_opts()
    Y = torch.zeros((q.n, XM_MAX_RANK), dtype=torch.float64, device=dev)
    R = torch.zeros((q.N, 3, 3), dtype=torch.float64, device=dev)
    s = torch.zeros((q.N,), dtype=torch.float64, device=dev)
    G = torch.zeros((q.N, 3, 3), dtype=torch.float64, device=dev)
    info = XmInfo()
    r_in = 0
    if Y0 is not None:
        Y0 = Y0.to(device=dev, dtype=torch.float64).contiguous()
        r_in = Y0.shape[1]
    allow = (XM_OK, XM_ENOTCERT, XM_ENOCONV) if allow_notcert else (XM_OK,)
    st = _check(lib().xm_solve(q.ctx.h, q.h, ctypes.byref(opts), r_in, _ptr(Y0), _ptr(Y), _ptr(R),
                               _ptr(s), _ptr(G), ctypes.byref(info)), allow)
    return dict(Y=Y, R=R, s=s, G=G, info=info.as_dict(), status=st)


def xm_certify(q: QMat, Y, opts: XmOpts | None = None):
    import torch
    dev = f"cuda:{q.ctx.device}"
    opts = opts or xm_default_opts()
    Y = Y.to(device=dev, dtype=torch.float64).contiguous()
    Lam = torch.zeros((q.N, 3, 3), dtype=torch.float64, device=dev)
    v = torch.zeros((q.n,), dtype=torch.float64, device=dev)
    info = XmInfo()
    _check(lib().xm_certify(q.ctx.h, q.h, ctypes.byref(opts), Y.shape[1], _ptr(Y), _ptr(Lam), _ptr(v),
                            ctypes.byref(info)))
    return dict(Lambda=Lam, v=v, info=info.as_dict())


def xm_backward(q: QMat, Y, rank: int, M: int, cam, lmk, ukp, w, dL_dG, opts: XmOpts | None = None,
                want_lambda: bool = False, allow_noconv: bool = False):
    """Adjoint of the certified optimum: (dL/du (E x 3), dL/dw (E), lambda or None, info, status)
    for a loss of G_i = Y_0 Y_i^T.  Y: n x ldy float64 CUDA tensor (xm_solve's Y), rank its
    used columns; dL_dG: N x 3 x 3 float64 CUDA tensor; observations as for xm_build_Q."""
    import torch
    dev = f"cuda:{q.ctx.device}"
    opts = opts or xm_default_opts()
    E = int(cam.shape[0])
    if Y.dtype != torch.float64 or Y.dim() != 2 or Y.shape[0] != q.n:
        raise ValueError(f"Y must be float64 of shape (n={q.n}, ldy)")
    if dL_dG.dtype != torch.float64 or tuple(dL_dG.shape) != (q.N, 3, 3):
        raise ValueError(f"dL_dG must be float64 of shape ({q.N}, 3, 3)")
    Y = Y.contiguous()
    dL_dG = dL_dG.contiguous()
    d_u = torch.empty((E, 3), dtype=torch.float64, device=dev)
    d_w = torch.empty((E,), dtype=torch.float64, device=dev)
    lam = torch.empty((q.n, rank), dtype=torch.float64, device=dev) if want_lambda else None
    info = XmAdjInfo()
    allow = (XM_OK, XM_ENOCONV) if allow_noconv else (XM_OK,)
    st = _check(lib().xm_backward(q.ctx.h, q.h, ctypes.byref(opts), rank, _ptr(Y), Y.shape[1], M, E,
                                  _ptr(cam), _ptr(lmk), _ptr(ukp), _ptr(w), _ptr(dL_dG), _ptr(d_u),
                                  _ptr(d_w), _ptr(lam), ctypes.byref(info)), allow)
    return d_u, d_w, lam, info.as_dict(), st


def xm_recover_tp(ctx: Context, N: int, M: int, cam, lmk, ukp, w, R, s, want_res2: bool = True):
    """(t (N x 3), p (M x 3), res2 (E) or None) of Eq. 7 for the rounded (R, s); CUDA tensors."""
    import torch
    dev = f"cuda:{ctx.device}"
    E = int(cam.shape[0])
    t = torch.empty((N, 3), dtype=torch.float64, device=dev)
    p = torch.empty((M, 3), dtype=torch.float64, device=dev)
    r2 = torch.empty((E,), dtype=torch.float64, device=dev) if want_res2 else None
    _check(lib().xm_recover_tp(ctx.h, N, M, E, _ptr(cam), _ptr(lmk), _ptr(ukp), _ptr(w),
                               _ptr(R.contiguous()), _ptr(s.contiguous()), _ptr(t), _ptr(p), _ptr(r2)))
    return t, p, r2


def xm_solve_xm2(ctx: Context, N: int, M: int, cam, lmk, ukp, w, opts: XmOpts | None = None,
                 drop_frac: float = 0.1, allow_notcert: bool = True):
    """XM^2 from observation tensors: dict(R, s, t, p, keep (bool, E), info_first, info_second,
    status)."""
    import torch
    dev = f"cuda:{ctx.device}"
    opts = opts or xm_default_opts()
    E = int(cam.shape[0])
    R = torch.zeros((N, 3, 3), dtype=torch.float64, device=dev)
    s = torch.zeros((N,), dtype=torch.float64, device=dev)
    t = torch.zeros((N, 3), dtype=torch.float64, device=dev)
    p = torch.zeros((M, 3), dtype=torch.float64, device=dev)
    keep = torch.zeros((E,), dtype=torch.uint8, device=dev)
    i1, i2 = XmInfo(), XmInfo()
    allow = (XM_OK, XM_ENOTCERT, XM_ENOCONV) if allow_notcert else (XM_OK,)
    st = _check(lib().xm_solve_xm2(ctx.h, N, M, E, _ptr(cam), _ptr(lmk), _ptr(ukp), _ptr(w), ctypes.byref(opts),
                                   drop_frac, _ptr(R), _ptr(s), _ptr(t), _ptr(p), _ptr(keep),
                                   ctypes.byref(i1), ctypes.byref(i2)), allow)
    return dict(R=R, s=s, t=t, p=p, keep=keep.bool(), info_first=i1.as_dict(), info_second=i2.as_dict(),
                status=st)


class Batch:
    """Owning handle of an xm_batch (dense per-scene copies of Q for the batched solve)."""

    def __init__(self, ctx: Context, qmats):
        self.ctx = ctx
        self.S = len(qmats)
        self.N = [q.N for q in qmats]
        arr = (_P * self.S)(*[q.h for q in qmats])
        h = _P()
        _check(lib().xm_batch_create(ctx.h, self.S, arr, ctypes.byref(h)))
        self.h = h

    def free(self):
        if getattr(self, "h", None):
            lib().xm_batch_free(self.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def xm_batch_create(ctx: Context, qmats) -> Batch:
    return Batch(ctx, qmats)


def xm_batch_autotune(b: Batch, reps: int = 8):
    """(rows per warp, column chunks per step) chosen for the four scene-size classes."""
    out = (ctypes.c_int * 8)()
    _check(lib().xm_batch_autotune(b.ctx.h, b.h, reps, out))
    return [(out[2 * k], out[2 * k + 1]) for k in range(4)]


def xm_batch_cluster(b: Batch, cs: int, n_min: int = 0) -> None:
    """Scenes with 3N >= n_min run on a thread-block cluster of cs CTAs (1, 2, 4); 0 for the
    automatic choice of either."""
    _check(lib().xm_batch_cluster(b.ctx.h, b.h, cs, n_min))


def xm_batch_launches(b: Batch) -> tuple:
    """(kernel launches per xm_solve_batched call, scenes on 4-CTA clusters) of the last solve's
    graph."""
    n = ctypes.c_int(0)
    q = ctypes.c_int(0)
    _check(lib().xm_batch_launches(b.ctx.h, b.h, ctypes.byref(n), ctypes.byref(q)))
    return n.value, q.value


def xm_solve_batched(b: Batch, opts: XmOpts | None = None, R=None, s=None, allow_notcert: bool = True):
    """Solves every scene; returns dict(R (sum N x 3 x 3), s (sum N), info (list of dicts), status).
    R and s may be passed in (float64 CUDA tensors) to reuse the captured graph."""
    import torch
    dev = f"cuda:{b.ctx.device}"
    opts = opts or xm_default_opts()
    tot = sum(b.N)
    R = torch.zeros((tot, 3, 3), dtype=torch.float64, device=dev) if R is None else R
    s = torch.zeros((tot,), dtype=torch.float64, device=dev) if s is None else s
    info = (XmBatchInfo * b.S)()
    allow = (XM_OK, XM_ENOTCERT, XM_ENOCONV) if allow_notcert else (XM_OK,)
    st = _check(lib().xm_solve_batched(b.ctx.h, b.h, ctypes.byref(opts), _ptr(R), _ptr(s), info), allow)
    return dict(R=R, s=s, info=[x.as_dict() for x in info], status=st)


def xm_pipeline_host(ctx: Context, N: int, M: int, cam, lmk, ukp, w, opts: XmOpts | None = None):
    """End to end from HOST numpy arrays (copies inside the call); returns (R, s, info, status)."""
    cam = np.ascontiguousarray(cam, dtype=np.int32)
    lmk = np.ascontiguousarray(lmk, dtype=np.int32)
    ukp = np.ascontiguousarray(ukp, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    R = np.zeros((N, 3, 3))
    s = np.zeros(N)
    info = XmInfo()
    opts = opts or xm_default_opts()
    st = _check(lib().xm_pipeline_host(ctx.h, N, M, cam.shape[0], cam.ctypes.data, lmk.ctypes.data,
                                       ukp.ctypes.data, w.ctypes.data, ctypes.byref(opts),
                                       R.ctypes.data, s.ctypes.data, ctypes.byref(info)),
                (XM_OK, XM_ENOTCERT, XM_ENOCONV))
    return R, s, info.as_dict(), st


def xm_pipeline_host_ptrs(ctx: Context, N: int, M: int, cam, lmk, ukp, w, opts: XmOpts, R_out, s_out):
    """xm_pipeline_host on (pinned) CPU torch tensors; R_out (N x 3 x 3) and s_out (N) are CPU
    float64 tensors written by the call.  Returns (info, status)."""
    import torch
    for t in (cam, lmk, ukp, w, R_out, s_out):
        if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
            raise TypeError("expected contiguous CPU tensors")
    info = XmInfo()
    st = _check(lib().xm_pipeline_host(ctx.h, N, M, cam.shape[0], cam.data_ptr(), lmk.data_ptr(),
                                       ukp.data_ptr(), w.data_ptr(), ctypes.byref(opts),
                                       R_out.data_ptr(), s_out.data_ptr(), ctypes.byref(info)),
                (XM_OK, XM_ENOTCERT, XM_ENOCONV))
    return info.as_dict(), st


def scene_tensors(sc, device: int = 0):
    """Observation arrays of a scene as CUDA tensors (cam, lmk, ukp, w)."""
    import torch
    dev = f"cuda:{device}"
    return (torch.as_tensor(sc.cam, dtype=torch.int32, device=dev),
            torch.as_tensor(sc.lmk, dtype=torch.int32, device=dev),
            torch.as_tensor(sc.ukp, dtype=torch.float64, device=dev).contiguous(),
            torch.as_tensor(sc.w, dtype=torch.float64, device=dev))

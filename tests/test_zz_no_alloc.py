"""xm_qy_noalloc: the sweep for callers that cannot let the library allocate device memory
(their memory is owned by their own pool allocator, or an allocation's implicit
synchronisation is not acceptable in their loop).  It keeps its padded operands in a fixed
device array inside the library; this checks it against xm_qy through the C ABI on two calls
in a row (the array keeps the previous call's contents), and that oversized requests are
rejected.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import EPS32, EPS64, ctx, gamma, rand_sym, torch

pytestmark = pytest.mark.gpu


def _noalloc(xm, C, q, prec, Y):
    W = torch.empty_like(Y)
    st = xm.lib().xm_qy_noalloc(C.h, q.h, prec, Y.shape[1], Y.data_ptr(), W.data_ptr())
    return st, W


def test_noalloc_sweep_matches_xm_qy_twice():
    from paper_2502_04640_b300 import xm
    C = ctx()
    try:
        Q1 = rand_sym(3 * 150, 11)                    # 450 rows: 4 tiles, ragged tail
        Q2 = rand_sym(3 * 61, 12)                     # smaller second call: stale rows must not leak
        q1 = xm.xm_qmat_from_dense(C, torch.tensor(Q1, device="cuda"))
        q2 = xm.xm_qmat_from_dense(C, torch.tensor(Q2, device="cuda"))
        rng = np.random.default_rng(5)
        # call 1: FP32, r = 4
        Y1 = torch.tensor(rng.standard_normal((450, 4)).astype(np.float32), device="cuda")
        st, W1 = _noalloc(xm, C, q1, xm.XM_FP32_BULK, Y1)
        assert st == xm.XM_OK
        ref1 = xm.xm_qy(q1, Y1, xm.XM_FP32_BULK)
        b1 = np.abs(Q1) @ np.abs(Y1.cpu().numpy().astype(np.float64))
        assert np.all(np.abs(W1.cpu().numpy() - ref1.cpu().numpy()) <= 2 * (EPS32 + gamma(452, EPS32)) * b1)
        # call 2: FP64, r = 3, on a smaller Q
        Y2 = torch.tensor(rng.standard_normal((183, 3)), device="cuda")
        st, W2 = _noalloc(xm, C, q2, xm.XM_FP64, Y2)
        assert st == xm.XM_OK
        ref2 = xm.xm_qy(q2, Y2, xm.XM_FP64)
        b2 = np.abs(Q2) @ np.abs(Y2.cpu().numpy())
        assert np.all(np.abs(W2.cpu().numpy() - ref2.cpu().numpy()) <= 2 * gamma(185, EPS64) * b2)
        torch.cuda.synchronize()
        q1.free(); q2.free()
    finally:
        C.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2502_04640_b300 import xm
    C = ctx()
    try:
        N = 11000                                      # n_pad = 33024: 2 * 33024 * 8 * 8 B > 4 MiB
        Qd = torch.zeros((3 * N, 3 * N), dtype=torch.float64, device="cuda")
        q = xm.xm_qmat_from_dense(C, Qd, xm.XM_STORE_FP64)
        del Qd
        Y = torch.zeros((3 * N, 8), dtype=torch.float64, device="cuda")
        st, _ = _noalloc(xm, C, q, xm.XM_FP64, Y)
        assert st == xm.XM_EINVAL
        assert b"scratch" in xm.lib().xm_last_error()
        q.free()
    finally:
        C.close()

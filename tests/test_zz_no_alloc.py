"""xm_qy_noalloc: the sweep for callers that cannot let the library allocate device memory
(their memory is owned by their own pool allocator, or an allocation's implicit
synchronisation is not acceptable in their loop).  It keeps its padded operands in a fixed
device array inside the library; this checks it against xm_qy through the C ABI on two calls
in a row (the array keeps the previous call's contents), and that oversized requests are
rejected.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import EPS32, EPS64, EPS_BF16, ctx, gamma, rand_sym, torch

pytestmark = pytest.mark.gpu


def _noalloc(xm, C, q, prec, Y):
    W = torch.empty_like(Y)
    st = xm.lib().xm_qy_noalloc(C.h, q.h, prec, Y.shape[1], Y.data_ptr(), W.data_ptr())
    return st, W


def test_noalloc_sweep_matches_xm_qy_twice():
    """Calls in a row on the same shared array, alternating between a 450-row and a 183-row Q (a
    smaller call after a larger one must not see stale rows), through every padded width
    (r = 1, the 4-column layout at r = 3 and 4, the 8-column layout at r = 6 and 8, which also
    moves W's offset in the array) and every storage precision (FP32, BF16, FP64)."""
    from paper_2502_04640_b300 import xm
    C = ctx()
    try:
        Q1 = rand_sym(3 * 150, 11)                    # 450 rows: 4 tiles, ragged tail
        Q2 = rand_sym(3 * 61, 12)                     # 183 rows: 2 tiles
        q1 = xm.xm_qmat_from_dense(C, torch.tensor(Q1, device="cuda"))
        q2 = xm.xm_qmat_from_dense(C, torch.tensor(Q2, device="cuda"))
        rng = np.random.default_rng(5)
        calls = [(q1, Q1, xm.XM_FP32_BULK, 4), (q2, Q2, xm.XM_FP64, 3), (q1, Q1, xm.XM_FP32_BULK, 6),
                 (q2, Q2, xm.XM_FP32_BULK, 1), (q1, Q1, xm.XM_BF16Q_BULK, 4), (q2, Q2, xm.XM_FP64, 8),
                 (q1, Q1, xm.XM_FP64, 1), (q2, Q2, xm.XM_BF16Q_BULK, 8)]
        for q, Qd, prec, r in calls:
            n = Qd.shape[0]
            if prec == xm.XM_FP64:
                Y = torch.tensor(rng.standard_normal((n, r)), device="cuda")
                eps = gamma(n + 2, EPS64)
            else:
                Y = torch.tensor(rng.standard_normal((n, r)).astype(np.float32), device="cuda")
                eps = (EPS_BF16 if prec == xm.XM_BF16Q_BULK else EPS32) + gamma(n + 2, EPS32)
            st, W = _noalloc(xm, C, q, prec, Y)
            assert st == xm.XM_OK
            ref = xm.xm_qy(q, Y, prec)
            b = np.abs(Qd) @ np.abs(Y.cpu().numpy().astype(np.float64))
            # both results are within the a-priori bound of the exact product, so of each other
            # within twice that bound
            assert np.all(np.abs(W.cpu().numpy() - ref.cpu().numpy()) <= 2 * eps * b), (prec, r)
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

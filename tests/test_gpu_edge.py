"""Degenerate inputs and host-side fault injection through the C ABI: a single camera (the
anchor alone, n = 3), a one-scene batch, a batch scene above the shared-memory limit, a NaN in a
caller-provided start point, and a zero time limit.  Every failure here is produced on the host
or by NaN arithmetic; none makes the GPU fault."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O
from tests.gpu_util import ctx, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


def _q(C, sc):
    from paper_2502_04640_b300 import xm
    return xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))


def test_single_camera_solve_is_trivially_certified(C):
    """N = 1: only the anchor, fixed to (I, 1) by the gauge (Sec. 2); Q vanishes (every landmark
    is seen once), f = 0 and the certificate holds with Z = 0."""
    from paper_2502_04640_b300 import xm
    sc = scenes.circle_scene(1, 20, 1, 0.0, seed=1)
    q = _q(C, sc)
    for prec in (0, 1):
        out = xm.xm_solve(q, xm.xm_default_opts(prec=prec), allow_notcert=False)
        assert out["info"]["certified"] == 1 and abs(out["info"]["f"]) <= 1e-12
        assert np.allclose(out["R"].cpu().numpy()[0], np.eye(3)) and out["s"].cpu().numpy()[0] == 1.0
    b = xm.xm_batch_create(C, [q])
    bo = xm.xm_solve_batched(b, xm.xm_default_opts(time_limit_s=10.0), allow_notcert=False)
    assert bo["info"][0]["certified"] == 1 and np.allclose(bo["R"].cpu().numpy()[0], np.eye(3))
    b.free()
    q.free()


def test_one_scene_batch_matches_single_solve(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.config1()
    q = _q(C, sc)
    single = xm.xm_solve(q, xm.xm_default_opts(), allow_notcert=False)
    b = xm.xm_batch_create(C, [q])
    bo = xm.xm_solve_batched(b, xm.xm_default_opts(time_limit_s=10.0), allow_notcert=False)
    assert abs(bo["info"][0]["f"] - single["info"]["f"]) <= 1e-6 * (1 + abs(single["info"]["f"]))
    assert np.abs(bo["R"].cpu().numpy() - single["R"].cpu().numpy()).max() <= 1e-5
    b.free()
    q.free()


def test_batch_scene_above_the_shared_memory_limit_is_rejected(C):
    """The batched solver stages a scene's whole sweep input and output in shared memory; 500
    cameras (3N = 1500) exceed the 227 KB of a CTA with the rank-8 kernel."""
    from paper_2502_04640_b300 import xm
    sc = scenes.circle_scene(500, 1000, 4, 0.01, seed=3)
    q = _q(C, sc)
    b = xm.xm_batch_create(C, [q])
    with pytest.raises(xm.XmError, match="XM_EINVAL"):
        xm.xm_solve_batched(b, xm.xm_default_opts())
    b.free()
    q.free()


def test_nan_start_point_reports_a_numeric_error(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.config1()
    q = _q(C, sc)
    Y0 = torch.tensor(O.initial_point(sc.N, 4), device="cuda")
    Y0[7, 1] = float("nan")
    with pytest.raises(xm.XmError, match="XM_ENUMERIC"):
        xm.xm_solve(q, xm.xm_default_opts(prec=0), Y0=Y0)
    # the context stays usable
    out = xm.xm_solve(q, xm.xm_default_opts(), allow_notcert=False)
    assert out["info"]["certified"] == 1
    q.free()


def test_zero_time_limit_returns_not_converged(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(40, 800, noise=0.02, seed=9)
    q = _q(C, sc)
    out = xm.xm_solve(q, xm.xm_default_opts(time_limit_s=1e-9))
    assert out["status"] == xm.XM_ENOCONV and out["info"]["certified"] == 0
    b = xm.xm_batch_create(C, [q])
    bo = xm.xm_solve_batched(b, xm.xm_default_opts(time_limit_s=1e-9))
    assert bo["status"] == xm.XM_ENOCONV and bo["info"][0]["status"] == xm.XM_ENOCONV
    b.free()
    q.free()


def test_bounded_wait_gives_up_and_the_context_stays_usable(C):
    """The pipelined kernels' waits are bounded polls of an mbarrier: a wait that nobody completes
    gives up after its limit, the kernel raises the timeout flag and the entry point returns
    XM_ETIMEOUT (no trap, nothing in flight); the same context then runs a sweep correctly."""
    from paper_2502_04640_b300 import xm
    assert xm.xm_selftest_wait(C, 1000, arrive=True) == xm.XM_OK
    assert xm.xm_selftest_wait(C, 1000, arrive=False) == xm.XM_ETIMEOUT
    assert b"bounded device wait" in xm.lib().xm_last_error()
    assert xm.xm_selftest_wait(C, 1, arrive=False) == xm.XM_ETIMEOUT
    assert xm.lib().xm_selftest_wait(C.h, 0, 0) == xm.XM_EINVAL
    assert xm.xm_selftest_wait(C, 1000, arrive=True) == xm.XM_OK     # the error word was cleared
    Q = np.random.default_rng(2).standard_normal((30, 30))
    Q = Q + Q.T
    q = xm.xm_qmat_from_dense(C, torch.tensor(Q, device="cuda"))
    Y = np.random.default_rng(3).standard_normal((30, 4))
    W = xm.xm_qy(q, torch.tensor(Y, device="cuda"), xm.XM_FP64).cpu().numpy()
    assert np.abs(W - Q @ Y).max() <= 1e-12 * np.abs(Q).sum()
    q.free()

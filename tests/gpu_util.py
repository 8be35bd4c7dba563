"""Shared helpers of the GPU tests (no method arithmetic: contexts, tolerances)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def ctx():
    from paper_2502_04640_b300 import xm
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return xm.Context(0)


def gamma(n, eps):
    """Rounding-error bound of an n-term dot product in any summation order: n eps / (1 - n eps)."""
    return n * eps / (1.0 - n * eps)


EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24
EPS_BF16 = 2.0 ** -8


def rand_sym(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return (A + A.T) / 2.0

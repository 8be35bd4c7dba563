"""The C-ABI library loads on a machine without a GPU and exports every symbol that
include/xm.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2502_04640_b300 import xm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "xm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xm_[a-z_0-9A-Z]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["xm_create", "xm_destroy", "xm_build_Q", "xm_qy", "xm_solve", "xm_certify",
                     "xm_free_Q", "xm_pipeline_host", "xm_last_error"]:
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    if not os.path.exists(xm.LIB_PATH):
        from paper_2502_04640_b300 import build
        build.build()
    L = xm.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert L.xm_abi_version() == 3


def test_default_opts_and_errors_without_device():
    o = xm.xm_default_opts()
    assert o.r0 == 4 and o.r_max == xm.XM_MAX_RANK and o.cert_tau_rel == 1e-6
    # every default the header documents for xm_opts
    documented = dict(prec=xm.XM_FP32_BULK, grad_tol_rel=1e-11, bulk_tol_rel=1e-9, max_outer=300,
                      max_tcg=200, max_polish=20, lanczos_max=800, lanczos_tol=1e-8,
                      time_limit_s=0.0, seed=12345, verbose=0, init_jitter=0.1, scale_reg=0.0,
                      precond=2, bulk_stall=-1, cert_lobpcg=1)
    for field, value in documented.items():
        assert getattr(o, field) == value, field
    L = xm.lib()
    # NULL arguments are rejected on the host before any device work
    assert L.xm_solve(None, None, None, 0, None, None, None, None, None, None) == xm.XM_EINVAL
    assert b"NULL" in L.xm_last_error()
    h = ctypes.c_void_p()
    st = L.xm_create(ctypes.byref(h), 0, None)
    assert st != xm.XM_OK or h.value    # no GPU here: a status, never a crash
    if st == xm.XM_OK:
        L.xm_destroy(h)


def test_library_needs_no_vendor_math_library():
    """Every kernel on the path is this library's own: libxm.so links the CUDA runtime only
    (no cuBLAS, cuSOLVER or other vendor math library among its dynamic dependencies)."""
    import shutil
    import subprocess
    if not os.path.exists(xm.LIB_PATH):
        from paper_2502_04640_b300 import build
        build.build()
    readelf = shutil.which("readelf")
    if readelf is None:
        import pytest
        pytest.skip("readelf not available")
    out = subprocess.run([readelf, "-d", xm.LIB_PATH], capture_output=True, text=True, check=True).stdout
    needed = re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out)
    assert needed, out
    vendor = [n for n in needed if re.match(r"lib(cublas|cublasLt|cusolver|cusparse|cufft|curand|cudnn)", n)]
    assert not vendor, needed

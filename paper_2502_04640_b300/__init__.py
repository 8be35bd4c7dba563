"""XM on B300: the Q.Y hot path, RTR-tCG, dual certificate and rounding as CUDA kernels
behind the C ABI of include/xm.h.  ``paper_2502_04640_b300.xm`` is the Python binding."""

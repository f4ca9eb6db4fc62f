"""GB300-native nested twisted frequency-filtering preconditioned CG
(arXiv 1909.09771).  The compute path is the CUDA library libffp.so (C ABI in
include/ffp.h); ``paper_1909_09771_gb300.ffp`` is its thin ctypes binding and
``paper_1909_09771_gb300.inputs`` draws the seeded synthetic workloads."""
__all__ = ["ffp", "inputs"]

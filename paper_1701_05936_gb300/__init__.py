"""GB300-native hot path of the pathwise lasso / elastic-net solver with
hybrid safe-strong (SSR-BEDPP) screening, after "The biglasso Package"
(Zeng & Breheny).

``paper_1701_05936_gb300.bl`` is the ctypes binding of the C-ABI library
``libbl.so`` (declared in ``include/biglasso_gpu.h``); every step of the path
runs in that library's CUDA kernels.  ``paper_1701_05936_gb300.synth`` holds
the seeded synthetic input generators.
"""
__all__ = ["bl", "synth"]

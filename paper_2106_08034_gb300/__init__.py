"""GB300-native weighted recursive least squares (wRLS) temporal denoiser for
volumetric path-traced frames (Iglesias-Guitian, Mane, Moon, "Real-Time Denoising of
Volumetric Path Tracing for Direct Volume Rendering", IEEE TVCG 2020, Sec. 5).

The compute path is the CUDA library ``libwrls.so`` (C ABI in ``include/wrls.h``);
``paper_2106_08034_gb300.wrls`` is its thin ctypes binding. Importing this package
loads nothing; the library is loaded on first use of the binding and raises if it
has not been built.
"""

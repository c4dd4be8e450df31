"""GB300-native engine for theoretical Rayleigh-wave dispersion curves
(the forward problem of MASW inversion, Kump & Martin, MASWAccelerated).

The compute path is the CUDA library ``libmasw`` (C ABI, ``include/masw.h``);
``paper_2003_02256_gb300.masw`` is its thin ctypes binding. Importing this
package does not load the library; the first API call does, and fails loudly
when it is missing.
"""
__all__ = ["masw", "workloads"]

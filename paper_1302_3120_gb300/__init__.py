"""GB300-native compressed-sensing SAR imaging with a chirp-scaling approximated
observation: the ITA hot path X <- T(X + mu M(S . (Y - G(X)))) in hand-written
sm_103a CUDA kernels behind the C ABI of include/csar.h.

``paper_1302_3120_gb300.csar`` is the ctypes binding (importing it requires the
built library ``libcsar.so``; ``paper_1302_3120_gb300.build.build()`` makes it).
"""
__all__ = ["build", "csar"]

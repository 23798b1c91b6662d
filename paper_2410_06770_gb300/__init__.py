"""GB300-native (sm_103a) xGETT: binary tensor contraction behind the BLAS-like
call of arXiv 2410.06770.

The compute path is the C-ABI library `libgett.so` built from `csrc/`; the
Python module `gett` is a thin ctypes binding to it (argument marshalling
only).  `synth` holds the seeded input generators.
"""
__all__ = ["synth"]

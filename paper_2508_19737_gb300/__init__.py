"""InfraredGP feed-forward propagation (FFP) on one GB300 (sm_103a).

The compute path lives in the CUDA library ``csrc/`` builds (``libigp.so``);
``api`` is a thin ctypes binding over its C-ABI (``include/igp.h``). Importing
this package loads nothing; the library is loaded on first use by ``api`` and
raises if it is missing.
"""
__version__ = "0.1.0"

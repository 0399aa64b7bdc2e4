"""FP64 CPU oracle for the InfraredGP feed-forward propagation (FFP).

TEST INFRASTRUCTURE ONLY. This package is the slow, plain reference that the
CUDA path is checked against. Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it. The
product library never imports, links or calls anything in here, and nothing in
here imports the product library: the two share no code.

Modules:
  fp64    -- CSR construction, Eq. 1 degree correction, Eq. 3 convolution,
             Eq. 4 layers, Alg. 1 / Alg. 2 drivers, BF16-storage emulation.
  philox  -- Philox4x64-10 counter-based generator and the Box-Muller map that
             turn (seed, row, column) into the random input Theta of Alg. 1.
  cluster -- the library's K-agnostic clusterer (BIRCH's leaf level, batched), the
             step that turns embeddings into blocks (Alg. 1, Alg. 2).
"""
from .fp64 import *  # noqa: F401,F403
from .philox import philox4x64_10, theta_input, uniforms_from_words, box_muller  # noqa: F401
from .cluster import CFState, cf_cluster, cf_predict  # noqa: F401

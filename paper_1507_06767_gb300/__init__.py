"""GB300 lattice Boltzmann step with the Knudsen refinement sensor (arXiv 1507.06767).

The computation lives in the CUDA library ``_build/liblbm.so`` (C ABI: ``include/lbm.h``); this
package is its Python binding.  Build the library with ``paper_1507_06767_gb300.build.build()``.
"""
from .lbm import *  # noqa: F401,F403
from .lbm import Lattice, LbmError, exported_symbols  # noqa: F401

"""GB300 library for Fourier-domain light-pollution maps (arXiv:1907.02891).

The compute path is ``liblp.so`` (hand-written sm_103a CUDA behind the C ABI
of ``include/lp.h``); ``lp`` is its thin ctypes binding and ``build`` compiles
it in-tree.  Importing the package loads nothing; the binding loads the
library on first use and fails loudly if it has not been built.
"""

__all__ = ["lp", "build"]

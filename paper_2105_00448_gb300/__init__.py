"""GB300 (sm_103a) library for the data-parallel hot path of one step of the
hybrid cellular automaton model of arXiv:2105.00448.

The compute path is ``libhca.so`` (CUDA kernels behind the C ABI of
``include/hca.h``); ``hca`` is its thin ctypes binding.  Importing this
package does not load the library; ``hca.load()`` does, and raises if the
library is missing or cannot be loaded.
"""

from . import hca  # noqa: F401

__all__ = ["hca"]

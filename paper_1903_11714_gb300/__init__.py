"""GB300-native checkerboard Metropolis sweep of the 2D Ising model.

The compute path is the CUDA library ``csrc/`` builds (``libising_gb300.so``,
C-ABI in ``include/ising.h``); ``ising`` is its ctypes binding.  Importing this
package does not load the library; ``ising.lib()`` does, and raises if the
library has not been built.
"""
__all__ = ["ising", "workloads"]

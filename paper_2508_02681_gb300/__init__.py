"""GB300 (sm_103a) UNO-CG: preconditioned CG with a unitary-neural-operator preconditioner for
periodic voxel homogenization (thermal c = 1, elastic c = 3).

The compute path is the CUDA library ``libunocg.so`` (C ABI in ``include/unocg.h``); this
package is its thin Python binding.  Importing the package does not load the library;
the first call does, and fails loudly if it is missing.
"""
from . import _lib  # noqa: F401
from ._lib import UnocgError  # noqa: F401

__all__ = ["api", "solver", "build", "UnocgError"]

"""GB300-native (sm_103a) iterative CMB map-making with two-level preconditioning.

The compute lives in ``libmapmaker.so`` (C ABI in include/mapmaker.h); this
package holds its build script and a ctypes binding.  Importing the package
does not load the library; ``mapmaker.load_library()`` (or creating a
``mapmaker.Context``) does, and raises if the library has not been built.
"""
from . import mapmaker  # noqa: F401
from .mapmaker import (Context, MapMakerError, MM_FP64, MM_FP32_MIXED, MM_PRECOND_BD,  # noqa: F401
                       MM_PRECOND_2L, load_library, estimate_bytes)

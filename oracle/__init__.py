"""FP64 CPU oracle for two-level preconditioned PCG map-making.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the CUDA path computes, written from the paper (Puglisi et
al., "Iterative map-making with two-level preconditioning for polarized CMB
data sets").  Only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may import it; the library itself never does, and shares no
code with it.

Every function is numpy in float64 and cites the passage it follows.  Pins
that tie it to something other than itself live in tests/test_oracle_pins.py.
Parity unpinned: none of the functions here; the paper's own iteration counts
(Sect. 7) are qualitative and are not used as pins.
"""
from .mapmaking import *  # noqa: F401,F403
from .mapmaking import __all__ as _all_mm
from .templates import *  # noqa: F401,F403
from .templates import __all__ as _all_t

__all__ = list(_all_mm) + list(_all_t)

"""CPU oracle for the FFT-Galerkin homogenization path (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU baseline use this
package.  It never imports the CUDA library, and the library never imports it.
"""
from .galerkin import *  # noqa: F401,F403
from .galerkin import __all__  # noqa: F401

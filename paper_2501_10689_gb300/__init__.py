"""GB300-native Kaczmarz-type RZF precoders (libkzprecode) and their Python binding.

The compute path is the CUDA library built from ``csrc/`` for sm_103a; this
package only loads it (``kzprecode``) and wraps it for autograd
(``autograd``).  Importing the package does not load the library; the first
call does, and raises if it has not been built.
"""
from . import kzprecode  # noqa: F401
from .kzprecode import KzError, precode, plan_from_instance, rhs_tensor  # noqa: F401

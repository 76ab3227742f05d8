"""GB300-native hybrid depth-of-field pass (Tan et al., arXiv 2210.06158).

The compute path is libdof.so (hand-written sm_103a CUDA behind the C ABI in
include/dof.h); `dof` is its ctypes binding.
"""

from . import dof  # noqa: F401
from ._build import build  # noqa: F401

"""GB300-native Liouville-Lanczos TDDFPT hot path (turboEELS method): the Liouvillian
applied to batches of plane-wave response orbitals and the Lanczos recursions that give
chi(Q, omega) and the loss function, as hand-written sm_103a CUDA kernels behind the C ABI
of include/ll.h.  `ll` is the ctypes binding; `build` compiles the library in-tree."""
from .build import build_library, LIB_PATH  # noqa: F401

"""tdlz: Liouville-Lanczos spin susceptibility on one GB300 (sm_103a).

The hot path of the paper's method -- the Liouvillian of the batch
representation applied to noncollinear spinor response orbitals at momentum q,
inside the non-Hermitian and pseudo-Hermitian Lanczos recursions, and chi(q, w)
from the resulting tridiagonal matrix -- runs in the CUDA library built from
``csrc/`` and declared in ``include/tdlz.h``.  ``binding`` is its ctypes
marshalling layer.
"""

from .binding import (Chain, Context, TdlzError, load_library, library_path,  # noqa: F401
                      TDLZ_FP64, TDLZ_MIXED, FLAVORS)
from .build_ext import build  # noqa: F401

"""Seeded synthetic inputs shared by the oracle and the GPU path.

This package stands in for the plane-wave ground-state code that precedes the
linear-response method (Sec. 3.1 of the paper: the occupied spinor states,
energies and densities are read from a previous SCF run).  It builds a model
noncollinear Hamiltonian (kinetic + local + exchange field + Kleinman-Bylander
projectors with spin-orbit, Eq. H0_k_plus_q), diagonalises it, and writes the
ground-state bundle.  It also draws the seeded random response vectors used by
the parity tests.

It holds none of the Liouvillian / Lanczos / spectrum arithmetic: those live,
independently, in ``oracle/`` (CPU, FP64) and in the CUDA library.
"""

from .model import GroundState, HA_MEV  # noqa: F401
from .configs import CONFIGS, make_ground_state  # noqa: F401
from .vectors import random_br_vector  # noqa: F401

"""Seeded random response vectors in the batch-representation layout.

Layout (X,Y sides) x k x band x spinor x plane wave: shape (2, nk, nocc, 2, npwx),
complex128, zero beyond npw_kq[k] (the k+q sphere of each k).
"""

from __future__ import annotations

import numpy as np


def random_br_vector(gs, seed: int = 7) -> np.ndarray:
    rng = np.random.default_rng(seed)
    shape = gs.br_shape
    v = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    for k in range(gs.nk):
        v[:, k, :, :, gs.npw_kq[k]:] = 0.0
    return v

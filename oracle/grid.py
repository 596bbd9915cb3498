"""Plane-wave sphere <-> real-space grid maps (oracle; FP64).

psi_s(r_j) = Omega^{-1/2} sum_{g in sphere} c[s][g] exp(+i G_g . r_j)
f(G)       = (Omega^{1/2} / Nr) sum_j f(r_j) exp(-i G . r_j)   (restricted to a sphere)

These are the discrete maps of a plane-wave code (the FFT, scipy.fft, is used as a
library primitive).  The flat grid index of Miller m is ((m1 mod n1) n2 + m2 mod n2) n3 + m3 mod n3.
"""

from __future__ import annotations

import numpy as np
import scipy.fft

# FFT worker threads (the library primitive runs on every host core)
WORKERS = -1


def flat_index(miller: np.ndarray, fft) -> np.ndarray:
    n1, n2, n3 = fft
    m = np.asarray(miller, dtype=np.int64)
    return ((m[:, 0] % n1) * n2 + (m[:, 1] % n2)) * n3 + (m[:, 2] % n3)


def fftn(a: np.ndarray) -> np.ndarray:
    """Unnormalised forward 3-D DFT, sum_j a_j exp(-i G.r_j)."""
    return scipy.fft.fftn(a, workers=WORKERS)


def ifftn(a: np.ndarray) -> np.ndarray:
    """Inverse 3-D DFT with the 1/Nr factor, (1/Nr) sum_G a_G exp(+i G.r_j)."""
    return scipy.fft.ifftn(a, workers=WORKERS)


def sphere_to_real(c: np.ndarray, idx: np.ndarray, fft, omega: float) -> np.ndarray:
    """c: (..., npw) sphere coefficients -> (..., Nr) grid values."""
    nr = int(np.prod(fft))
    lead = c.shape[:-1]
    g = np.zeros(lead + (nr,), dtype=np.complex128)
    g[..., idx] = c
    g = g.reshape(lead + tuple(fft))
    axes = tuple(range(len(lead), len(lead) + 3))
    return scipy.fft.ifftn(g, axes=axes, workers=WORKERS).reshape(lead + (nr,)) * (nr / np.sqrt(omega))


def real_to_sphere(f: np.ndarray, idx: np.ndarray, fft, omega: float) -> np.ndarray:
    """f: (..., Nr) grid values -> (..., npw) coefficients on the sphere idx."""
    nr = int(np.prod(fft))
    lead = f.shape[:-1]
    axes = tuple(range(len(lead), len(lead) + 3))
    g = scipy.fft.fftn(f.reshape(lead + tuple(fft)), axes=axes, workers=WORKERS).reshape(lead + (nr,))
    return g[..., idx] * (np.sqrt(omega) / nr)


def grid_millers(fft) -> np.ndarray:
    ax = [np.fft.fftfreq(n, d=1.0 / n).astype(np.int64) for n in fft]
    a, b, c = np.meshgrid(*ax, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)

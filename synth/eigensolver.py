"""Lowest eigenpairs of the model Hamiltonian.

Small problems: dense ``numpy.linalg.eigh``.  Larger problems: block LOBPCG
(Knyazev 2001) with a kinetic-energy preconditioner on the matrix-free FFT
application, in torch so that it runs on CPU or on a GPU when one is present.
This is input generation (the stand-in for the SCF code's Davidson solver), not
part of the linear-response method.
"""

from __future__ import annotations

import numpy as np


def dense_lowest(h: np.ndarray, nev: int):
    w, v = np.linalg.eigh(h)
    return w[:nev], v[:, :nev]


def _eigh_small(t, a):
    """Eigen-decomposition of a small Hermitian matrix on the host (GPU eigh is slow here)."""
    w, v = t.linalg.eigh(0.5 * (a + a.conj().T).cpu())
    return w.to(a.device), v.to(a.device)


def _orthonormal(t, s, drop=1e-10):
    """Orthonormal basis of span(s) (eigen-decomposition of the scaled Gram matrix)."""
    g = s.conj().T @ s
    d = t.rsqrt(t.clamp(t.real(t.diagonal(g)), min=1e-300))
    g = d[:, None] * g * d[None, :]
    lam, v = _eigh_small(t, g)
    keep = lam > drop * lam.max()
    return s @ ((d[:, None] * v[:, keep]) * t.rsqrt(lam[keep])[None, :])


def lobpcg(t, apply_h, kin, x0, nconv, tol=1e-9, maxiter=400, log=None):
    """Block LOBPCG on vectors stored as columns of an (n, m) complex128 tensor.

    Each iteration: residuals R = HX - X Theta, preconditioned W = K R with
    K = 1 / (1 + kin / e_ref); the search block Z = [W, P] is orthonormalised
    against X and H is applied to it afresh (no recurrence for HP, which keeps
    the Rayleigh-Ritz data accurate near convergence); P is the Z-part of the new
    Ritz vectors.  Returns (theta[:m], X, residual norms).
    """
    m = x0.shape[1]
    x = _orthonormal(t, x0)
    hx = apply_h(x)
    a = x.conj().T @ hx
    theta, c = _eigh_small(t, a)
    x, hx = x @ c, hx @ c
    p = None
    e_ref = max(1.0, float(t.mean(kin)))
    prec = 1.0 / (1.0 + kin / e_ref)
    res = None
    for it in range(maxiter):
        r = hx - x * theta[None, :]
        res = t.linalg.vector_norm(r, dim=0)
        if log is not None and it % 20 == 0:
            log(f"  lobpcg it {it}: max resid {float(res[:nconv].max()):.3e}")
        if float(res[:nconv].max()) < tol:
            break
        z = prec[:, None] * r
        if p is not None:
            z = t.cat([z, p], 1)
        for _ in range(2):
            z = z - x @ (x.conj().T @ z)
        z = _orthonormal(t, z)
        hz = apply_h(z)
        s, hs = t.cat([x, z], 1), t.cat([hx, hz], 1)
        a = s.conj().T @ hs
        th, c = _eigh_small(t, a)
        p = z @ c[m:, :m]
        x, hx, theta = s @ c[:, :m], hs @ c[:, :m], th[:m]
    hx = apply_h(x)
    r = hx - x * theta[None, :]
    res = t.linalg.vector_norm(r, dim=0)
    return theta, x, res

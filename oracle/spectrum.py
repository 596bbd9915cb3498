"""chi(omega) from Lanczos coefficients (oracle; FP64).

Eqs. resolvent_Liouvillian_Lanczos_q and post_processing: solve
(omega + i eta - T) eta_vec = e_1 for each frequency (Lorentzian broadening
omega -> omega + i eta) and take chi_{lambda mu} = w n0 sum_i conj(z^lambda_i) eta_vec_i.
The factor w n0 restores the start-vector norm and the k weight that the
printed formula leaves implicit (reading).  Frequencies in Hartree here;
1 Ha = 27211.386245988 meV.

``chi_thomas`` uses plain Thomas elimination; ``chi_banded`` re-solves with the
pivoted banded LAPACK routine as an independent check.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg

HA_MEV = 27211.386245988


def tridiag_parts(alpha, beta, gamma, m):
    d = np.asarray(alpha[:m], dtype=np.complex128)
    lower = np.asarray(beta[:m - 1], dtype=np.complex128)  # T_{j+1,j}
    upper = np.asarray(gamma[:m - 1], dtype=np.complex128)  # T_{j,j+1}
    return d, lower, upper


def solve_thomas(zdiag, lower, upper):
    """Solve A x = e_1 for tridiagonal A by Thomas elimination (no pivoting).

    zdiag: (m, nw) diagonals for nw right-hand sides solved side by side;
    lower[j] = A[j+1, j], upper[j] = A[j, j+1] (shared by all columns).
    """
    m = zdiag.shape[0]
    cp = np.zeros_like(zdiag)
    yp = np.zeros_like(zdiag)
    piv = zdiag[0]
    if m > 1:
        cp[0] = upper[0] / piv
    yp[0] = 1.0 / piv
    for j in range(1, m):
        piv = zdiag[j] - lower[j - 1] * cp[j - 1]
        if j < m - 1:
            cp[j] = upper[j] / piv
        yp[j] = (0.0 - lower[j - 1] * yp[j - 1]) / piv
    x = np.zeros_like(zdiag)
    x[m - 1] = yp[m - 1]
    for j in range(m - 2, -1, -1):
        x[j] = yp[j] - cp[j] * x[j + 1]
    return x


def chi_thomas(coef, omegas, eta, w, m=None):
    """chi[lambda, iw] for one chain (Hartree units for omegas and eta)."""
    m = coef.steps if m is None else m
    d, lo, up = tridiag_parts(coef.alpha, coef.beta, coef.gamma, m)
    om = np.asarray(omegas, dtype=np.float64)
    zdiag = (om[None, :] + 1j * eta) - d[:, None]
    x = solve_thomas(zdiag, -lo, -up)  # (m, nw)
    return w * coef.n0 * (coef.z[:, :m].conj() @ x)


def chi_banded(coef, omegas, eta, w, m=None):
    m = coef.steps if m is None else m
    d, lo, up = tridiag_parts(coef.alpha, coef.beta, coef.gamma, m)
    out = np.zeros((coef.z.shape[0], len(omegas)), dtype=np.complex128)
    e1 = np.zeros(m, dtype=np.complex128)
    e1[0] = 1.0
    for iw, om in enumerate(omegas):
        ab = np.zeros((3, m), dtype=np.complex128)
        ab[0, 1:] = -up
        ab[1, :] = (om + 1j * eta) - d
        ab[2, :-1] = -lo
        x = scipy.linalg.solve_banded((1, 1), ab, e1)
        out[:, iw] = w * coef.n0 * (coef.z[:, :m].conj() @ x)
    return out


def omega_grid_mev(start, end, step):
    n = int(np.floor((end - start) / step + 0.5)) + 1
    return start + step * np.arange(n)


def chi(coef, omegas, eta, w, m=None):
    """Primary oracle spectrum: the pivoted banded solve (robust for every flavour)."""
    return chi_banded(coef, omegas, eta, w, m)


# --------------------------------------------------------------- extrapolation
# Sec. 3.3 of the paper: the first itermax0 coefficients are the computed ones; up
# to itermax the chain is continued with extrapolated coefficients, either one
# constant ('constant') or two alternating constants ('osc', bi-constant), and the
# z coefficients are zero beyond itermax0.  Reading (the averaging window is not
# given): the constants are the means over the last half of the computed
# coefficients, [itermax0 // 2, itermax0), taken over all indices for 'constant'
# and separately over even and odd indices for 'osc'.

def extrapolation_constants(coef, itermax0, kind):
    """Returns {parity: (alpha, beta, gamma)} with parity 0/1 (same for 'constant')."""
    lo = itermax0 // 2
    idx = np.arange(lo, itermax0)
    out = {}
    for parity in (0, 1):
        sel = idx if kind == "constant" else idx[idx % 2 == parity]
        out[parity] = (np.mean(coef.alpha[sel]), np.mean(coef.beta[sel]),
                       np.mean(coef.gamma[sel]))
    return out


def extend_coefficients(coef, itermax0, itermax, kind):
    """Explicitly extended coefficient arrays of length itermax."""
    import dataclasses
    if kind == "no" or itermax <= itermax0:
        m = min(itermax0, coef.steps)
        return dataclasses.replace(coef, alpha=coef.alpha[:m], beta=coef.beta[:m],
                                   gamma=coef.gamma[:m], z=coef.z[:, :m], steps=m)
    if itermax0 > coef.steps:
        raise ValueError("itermax0 exceeds the computed coefficients")
    c = extrapolation_constants(coef, itermax0, kind)
    al = np.zeros(itermax, dtype=np.complex128)
    be = np.zeros(itermax)
    ga = np.zeros(itermax, dtype=np.complex128)
    z = np.zeros((coef.z.shape[0], itermax), dtype=np.complex128)
    al[:itermax0] = coef.alpha[:itermax0]
    # beta[j] (= beta_{j+2}) links steps j and j+1; the chain computed it for
    # j < itermax0 (its last step yields the link to the first extrapolated step)
    be[:itermax0] = coef.beta[:itermax0]
    ga[:itermax0] = coef.gamma[:itermax0]
    z[:, :itermax0] = coef.z[:, :itermax0]
    for j in range(itermax0, itermax):
        al[j] = c[j % 2][0]
        be[j] = c[j % 2][1].real
        ga[j] = c[j % 2][2]
    return dataclasses.replace(coef, alpha=al, beta=be, gamma=ga, z=z, steps=itermax)


def chi_extrapolated(coef, omegas, eta, w, itermax0, itermax, kind):
    """chi from the explicitly extended tridiagonal system (pivoted banded solve)."""
    ext = extend_coefficients(coef, itermax0, itermax, kind)
    return chi_banded(ext, omegas, eta, w)


def structure_factor(chi3, q):
    """S(q, omega) = -Im Tr[P_perp(q) chi(q, q; omega)] (Eq. S_def, Sec. 2.1), with
    P_perp_ab = delta_ab - q_a q_b / q^2 and chi3[mu][lambda][w] = chi_{lambda mu}(w)
    (the chi rows of the chains mu = x, y, z).  Tr[P chi] = sum_ab P_ab chi_ba."""
    q = np.asarray(q, dtype=np.float64)
    p = np.eye(3) - np.outer(q, q) / (q @ q)
    chi3 = np.asarray(chi3, dtype=np.complex128)
    s = np.zeros(chi3.shape[-1], dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            s += p[a, b] * chi3[a, b]  # chi_ba is row b of chain a
    return -s.imag

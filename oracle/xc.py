"""Adiabatic LSDA response kernel (oracle; FP64).

Eqs. v_XC_q and b_XC_q of the paper: the response XC potentials are the second
derivatives of the LSDA energy density e_xc(n, |m|) taken at the ground-state
(n0, m0) and contracted with (n', m').  With rho = (n, m_x, m_y, m_z) (Pauli
units: the Bohr magneton is factored out of both m' and the potential) the 4x4
symmetric kernel is f_ab = d^2 e / d rho_a d rho_b.

Functional: Slater exchange in its spin-polarised form,
    e_x(n_up, n_dn) = -(3/4) (6/pi)^{1/3} (n_up^{4/3} + n_dn^{4/3}),
    n_up/dn = (n +- |m|) / 2,
so v_s = -(6 n_s / pi)^{1/3} and f_s = d v_s / d n_s = -(1/3) (6/pi)^{1/3} n_s^{-2/3}.
Chain rule through |m| (m_hat = m/|m|):
    f_00 = (f_up + f_dn)/4
    f_0i = (f_up - f_dn)/4 m_hat_i
    f_ij = (f_up + f_dn)/4 m_hat_i m_hat_j + (v_up - v_dn)/(2|m|) (delta_ij - m_hat_i m_hat_j)

Thresholds (the paper gives none for this model): f = 0 where n < 1e-10;
n_up, n_dn floored at 1e-4 before the derivatives; where |m| < 1e-12 n the
transverse factor takes its |m| -> 0 limit f(n/2)/2 and m_hat = z.
Output layout: 10 rows in the order 00,01,02,03,11,12,13,22,23,33.
"""

from __future__ import annotations

import numpy as np

C6PI = (6.0 / np.pi) ** (1.0 / 3.0)
N_MIN = 1e-10
NS_FLOOR = 1e-4
M_REL = 1e-12
PAIRS = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]


def slater_energy(n, mabs):
    nu = np.maximum(0.5 * (n + mabs), NS_FLOOR)
    nd = np.maximum(0.5 * (n - mabs), NS_FLOOR)
    return -0.75 * C6PI * (nu ** (4.0 / 3.0) + nd ** (4.0 / 3.0))


def kernel_table(n0: np.ndarray, m0: np.ndarray) -> np.ndarray:
    """(10, Nr) table of f_ab at every grid point."""
    nr = n0.shape[0]
    out = np.zeros((10, nr))
    for j in range(nr):
        f = point_kernel(float(n0[j]), m0[:, j])
        for p, (a, b) in enumerate(PAIRS):
            out[p, j] = f[a, b]
    return out


def point_kernel(n: float, m: np.ndarray) -> np.ndarray:
    """4x4 kernel at one point (plain scalar arithmetic)."""
    f = np.zeros((4, 4))
    if n < N_MIN:
        return f
    mabs = float(np.sqrt(m[0] ** 2 + m[1] ** 2 + m[2] ** 2))
    nu = max(0.5 * (n + mabs), NS_FLOOR)
    nd = max(0.5 * (n - mabs), NS_FLOOR)
    fu = -(1.0 / 3.0) * C6PI * nu ** (-2.0 / 3.0)
    fd = -(1.0 / 3.0) * C6PI * nd ** (-2.0 / 3.0)
    if mabs < M_REL * n:
        mh = np.array([0.0, 0.0, 1.0])
        trans = 0.5 * (-(1.0 / 3.0) * C6PI * max(0.5 * n, NS_FLOOR) ** (-2.0 / 3.0))
    else:
        mh = np.asarray(m, dtype=np.float64) / mabs
        vu = -(6.0 * nu / np.pi) ** (1.0 / 3.0)
        vd = -(6.0 * nd / np.pi) ** (1.0 / 3.0)
        trans = (vu - vd) / (2.0 * mabs)
    f[0, 0] = 0.25 * (fu + fd)
    for i in range(3):
        f[0, 1 + i] = f[1 + i, 0] = 0.25 * (fu - fd) * mh[i]
        for k in range(3):
            f[1 + i, 1 + k] = 0.25 * (fu + fd) * mh[i] * mh[k] + trans * ((i == k) - mh[i] * mh[k])
    return f


def apply_kernel(table: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """v_a(r) = sum_b f_ab(r) rho_b(r); rho: (4, Nr) complex."""
    out = np.zeros_like(rho)
    for p, (a, b) in enumerate(PAIRS):
        out[a] += table[p] * rho[b]
        if a != b:
            out[b] += table[p] * rho[a]
    return out

"""Lanczos recursions for chi_{lambda mu} = (u^lambda, (omega - L)^{-1} v^mu) (oracle; FP64).

Sec. 2.5 of the paper names two flavours; both build a tridiagonal T with
diagonal alpha_j, sub-diagonal T_{j+1,j} = beta_{j+1} and super-diagonal
T_{j,j+1} = gamma_{j+1}, and record z_j = (q_j, u^lambda) = q_j^H u^lambda on the
fly.  chi is then w * n0 * z^H (omega - T)^{-1} e_1 (see ``spectrum``).

* Non-Hermitian biorthogonalisation: q_1 = p_1 = v / ||v||; two chains with L
  and L^H (= J L J), (T)_ij = (p_i, L q_j); two L applications per step.
* Pseudo-Hermitian, J metric ("ph"): L is self-adjoint in the indefinite
  metric J (L^H J = J L); one L application per step; |gamma| = beta, signs
  from the J-norms (the paper's remark that gamma equals beta up to a sign).
* Pseudo-Hermitian, positive-definite metric ("phm"): L = J (D + K) is
  self-adjoint in <a, b>_M = a^H (D + K) b = a^H J L b, a standard Hermitian
  Lanczos with a modified scalar product.  alpha_j = (L q_j)^H J (L q_j) needs
  no extra product; the norm of the next residual r needs L r, which is the
  next step's product, so the normalisation lags one product behind and the
  chain still costs one L per step.  T is real symmetric (gamma = beta).
  Requires D + K > 0 (a stable ground state); a non-positive M-norm stops the
  chain with status "indefinite".

Coefficient storage (0-based step j = 0..M-1 for the paper's j+1):
alpha[j] = alpha_{j+1}, beta[j] = beta_{j+2}, gamma[j] = gamma_{j+2}, z[l][j] = z_{j+1}.
Breakdown (|c| < 1e-14 ||r|| ||t||) truncates the chain; ``status`` says so.
"""

from __future__ import annotations

import dataclasses
import numpy as np

from .liouvillian import jdot, jmul

BREAKDOWN_TOL = 1e-14


@dataclasses.dataclass
class Coefficients:
    alpha: np.ndarray  # (M,) complex
    beta: np.ndarray  # (M,) real
    gamma: np.ndarray  # (M,) complex
    z: np.ndarray  # (3, M) complex
    n0: float
    steps: int
    status: str
    alpha_imag_max: float = 0.0
    basis_q: list = dataclasses.field(default_factory=list)  # first q_j when requested
    basis_p: list = dataclasses.field(default_factory=list)  # first p_j when requested
    signs: list = dataclasses.field(default_factory=list)  # PH: s_j = sign of q_j^H J q_j


def lanczos_ph(apply_l, v, u_list, nsteps, keep_basis=0):
    """Pseudo-Hermitian (J-metric) recursion; one L per step."""
    c0 = jdot(v, v).real
    n0 = float(np.sqrt(abs(c0)))
    s = 1.0 if c0 >= 0 else -1.0
    q = v / n0
    q_prev = np.zeros_like(v)
    gamma_j = 0.0
    al = np.zeros(nsteps, dtype=np.complex128)
    be = np.zeros(nsteps)
    ga = np.zeros(nsteps, dtype=np.complex128)
    z = np.zeros((len(u_list), nsteps), dtype=np.complex128)
    imag_max = 0.0
    status = "ok"
    steps = nsteps
    bq, sg = [], []
    for j in range(nsteps):
        if j < keep_basis:
            bq.append(q.copy())
            sg.append(s)
        a = apply_l(q)
        aj = s * jdot(q, a)
        imag_max = max(imag_max, abs(aj.imag))
        alpha = aj.real
        for li, u in enumerate(u_list):
            z[li, j] = np.vdot(q, u)
        r = a - alpha * q - gamma_j * q_prev
        c = jdot(r, r).real
        rn2 = np.vdot(r, r).real
        al[j] = alpha
        if abs(c) < BREAKDOWN_TOL * rn2 or rn2 == 0.0:
            status = "breakdown"
            steps = j + 1
            break
        beta_n = np.sqrt(abs(c))
        s_n = 1.0 if c >= 0 else -1.0
        gamma_n = s * s_n * beta_n
        be[j], ga[j] = beta_n, gamma_n
        q_prev, q = q, r / beta_n
        s, gamma_j = s_n, gamma_n
    return Coefficients(al[:steps], be[:steps], ga[:steps], z[:, :steps], n0, steps, status,
                        imag_max, bq, [sj * jmul(qj) for sj, qj in zip(sg, bq)], sg)


def lanczos_nh(apply_l, apply_lh, v, u_list, nsteps, keep_basis=0):
    """Non-Hermitian biorthogonal recursion; two L applications per step."""
    n0 = float(np.linalg.norm(v))
    q = v / n0
    p = q.copy()
    q_prev = np.zeros_like(v)
    p_prev = np.zeros_like(v)
    beta_j, gamma_j = 0.0, 0.0
    al = np.zeros(nsteps, dtype=np.complex128)
    be = np.zeros(nsteps)
    ga = np.zeros(nsteps, dtype=np.complex128)
    z = np.zeros((len(u_list), nsteps), dtype=np.complex128)
    status = "ok"
    steps = nsteps
    bq, bp = [], []
    for j in range(nsteps):
        if j < keep_basis:
            bq.append(q.copy())
            bp.append(p.copy())
        a = apply_l(q)
        b = apply_lh(p)
        alpha = np.vdot(p, a)
        for li, u in enumerate(u_list):
            z[li, j] = np.vdot(q, u)
        r = a - alpha * q - gamma_j * q_prev
        t = b - np.conj(alpha) * p - np.conj(beta_j) * p_prev
        c = np.vdot(t, r)
        al[j] = alpha
        if abs(c) < BREAKDOWN_TOL * np.linalg.norm(r) * np.linalg.norm(t) or abs(c) == 0.0:
            status = "breakdown"
            steps = j + 1
            break
        beta_n = np.sqrt(abs(c))
        gamma_n = c / beta_n
        be[j], ga[j] = beta_n, gamma_n
        q_prev, q = q, r / beta_n
        p_prev, p = p, t / np.conj(gamma_n)
        beta_j, gamma_j = beta_n, gamma_n
    return Coefficients(al[:steps], be[:steps], ga[:steps], z[:, :steps], n0, steps, status,
                        0.0, bq, bp)


def lanczos_phm(apply_l, v, u_list, nsteps, keep_basis=0):
    """Pseudo-Hermitian recursion in the positive-definite metric M = J L; one L per step."""
    r = np.array(v, dtype=np.complex128, copy=True)
    w = apply_l(r)
    c = jdot(r, w).real
    if c <= 0.0:
        return Coefficients(np.zeros(0, complex), np.zeros(0), np.zeros(0, complex),
                            np.zeros((len(u_list), 0), complex), 0.0, 0, "indefinite")
    n0 = float(np.sqrt(c))
    q, lq = r / n0, w / n0
    q_prev = np.zeros_like(r)
    beta_j = 0.0
    al = np.zeros(nsteps, dtype=np.complex128)
    be = np.zeros(nsteps)
    z = np.zeros((len(u_list), nsteps), dtype=np.complex128)
    status = "ok"
    steps = nsteps
    bq, bp = [], []
    for j in range(nsteps):
        if j < keep_basis:
            bq.append(q.copy())
            bp.append(jmul(lq))  # p_j = M q_j = J L q_j
        alpha = jdot(lq, lq).real
        for li, u in enumerate(u_list):
            z[li, j] = np.vdot(q, u)
        r = lq - alpha * q - beta_j * q_prev
        w = apply_l(r)
        c = jdot(r, w).real
        al[j] = alpha
        if c <= BREAKDOWN_TOL * np.linalg.norm(r) * np.linalg.norm(w):
            status = "breakdown" if c >= 0.0 else "indefinite"
            steps = j + 1
            break
        beta_n = float(np.sqrt(c))
        be[j] = beta_n
        q_prev, q, lq = q, r / beta_n, w / beta_n
        beta_j = beta_n
    return Coefficients(al[:steps], be[:steps], be[:steps].astype(np.complex128), z[:, :steps],
                        n0, steps, status, 0.0, bq, bp)


def run_chain(lv, mu, nsteps, flavor="ph", keep_basis=0, ncomp=3):
    """Chain for column mu of chi: start vector v^mu, left vectors u^x, u^y, u^z (and
    with ncomp = 4 the charge u^0 as the fourth, for the 4x4 susceptibility)."""
    v = lv.start_vector(mu)
    u = [lv.left_vector(l) for l in range(ncomp)]
    if flavor == "ph":
        return lanczos_ph(lv.apply, v, u, nsteps, keep_basis)
    if flavor == "phm":
        return lanczos_phm(lv.apply, v, u, nsteps, keep_basis)
    return lanczos_nh(lv.apply, lv.apply_adjoint, v, u, nsteps, keep_basis)

"""Brute-force particle-hole construction of the Liouvillian (test helper).

Independent of ``oracle.liouvillian``: the Hamiltonians are built as explicit
dense matrices (circular convolution with the grid Fourier coefficients of
v_loc and B, plus the projector sum), fully diagonalised, and the coupling
matrix is assembled from explicit DFT matrices, never from the oracle's maps.

Particle-hole basis e_(side,k,n,c): the empty eigenvector phi^side_{c,k+q}
placed in band slot n of the given side at k.  In that basis

    L = J (D + K),  D = diag(e_c(k+q) - e_n(k)),
    K_ab = w (Omega / Nr) sum_r tau_a(r)^H F tau_b(r),
    tau_(side,k,n,c),alpha(r) = t_alpha U_n(r)^dagger sigma_alpha phi_c(r),

with t = (1,1,1,1) on X and (1,-1,-1,-1) on Y, and F the Hartree (on alpha=0)
plus f_xc (pointwise 4x4) operator.
"""

from __future__ import annotations

import numpy as np

PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)
SIG4 = np.concatenate([np.eye(2, dtype=np.complex128)[None], PAULI])


def _grid_points(fft):
    ax = [np.arange(n) for n in fft]
    a, b, c = np.meshgrid(*ax, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def _centered_millers(fft):
    ax = [np.array([m if m < (n + 1) // 2 else m - n for m in range(n)]) for n in fft]
    a, b, c = np.meshgrid(*ax, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), c.ravel()], axis=1)


def dft_matrix(miller, fft):
    """E[j, g] = exp(+i G_g . r_j) = exp(2 pi i sum_d m_d j_d / n_d)."""
    pts = _grid_points(fft).astype(np.float64) / np.array(fft, dtype=np.float64)[None, :]
    return np.exp(2j * np.pi * (pts @ np.asarray(miller, dtype=np.float64).T))


def dense_h(gs, sign, p, miller, beta):
    fft = gs.fft
    nr = int(np.prod(fft))
    bvec = 2 * np.pi * np.linalg.inv(gs.lattice).T
    pts = _grid_points(fft).astype(np.float64) / np.array(fft, dtype=np.float64)[None, :]
    npw = miller.shape[0]
    # Fourier coefficient of a grid field at Miller difference d: (1/Nr) sum_j f_j e^{-i G_d r_j}
    dm = (miller[:, None, :] - miller[None, :, :]).reshape(-1, 3).astype(np.float64)
    uniq, inv = np.unique(dm, axis=0, return_inverse=True)
    phase = np.exp(-2j * np.pi * (pts @ uniq.T)) / nr  # (Nr, nuniq)
    vq = (gs.vloc @ phase)[inv].reshape(npw, npw)
    bq = [(gs.bfield[i] @ phase)[inv].reshape(npw, npw) for i in range(3)]
    h = np.kron(np.eye(2), vq).astype(np.complex128)
    for i in range(3):
        h += sign * np.kron(PAULI[i], bq[i])
    kg = p[None, :] + miller @ bvec
    h += np.diag(np.tile(0.5 * np.sum(kg * kg, axis=1), 2))
    for s in range(2):
        for t in range(2):
            h[s * npw:(s + 1) * npw, t * npw:(t + 1) * npw] += (
                beta.T @ gs.dnl[s::2, t::2] @ beta.conj())
    return h


def xc_matrix_from_table(table):
    pairs = [(0, 0), (0, 1), (0, 2), (0, 3), (1, 1), (1, 2), (1, 3), (2, 2), (2, 3), (3, 3)]
    f = np.zeros((4, 4, table.shape[1]))
    for p, (a, b) in enumerate(pairs):
        f[a, b] = table[p]
        f[b, a] = table[p]
    return f


class ParticleHole:
    def __init__(self, gs, fxc_table):
        self.gs = gs
        fft = gs.fft
        nr = int(np.prod(fft))
        self.nr = nr
        omega = abs(np.linalg.det(gs.lattice))
        self.omega = omega
        nb = gs.nocc
        self.blocks = []  # (side, k, phi (2npw, nemp), e_emp, U_occ_real (nb,2,Nr), phi_real)
        for side, sign in ((0, 1), (1, -1)):
            for k in range(gs.nk):
                mkq = gs.miller_kq[k, :gs.npw_kq[k]]
                mk = gs.miller_k[k, :gs.npw_k[k]]
                h = dense_h(gs, sign, gs.kpts[k] + gs.q, mkq, gs.beta_kq[k, :, :gs.npw_kq[k]])
                e, v = np.linalg.eigh(h)
                phi = v[:, nb:]
                npw = mkq.shape[0]
                ekq = dft_matrix(mkq, fft) / np.sqrt(omega)
                ek = dft_matrix(mk, fft) / np.sqrt(omega)
                phir = np.stack([ekq @ phi[:npw], ekq @ phi[npw:]], axis=0)  # (2, Nr, nemp)
                cu = gs.coeff_k[side, k, :, :, :gs.npw_k[k]]
                ur = np.einsum("rg,nsg->nsr", ek, cu)
                self.blocks.append(dict(side=side, k=k, phi=phi, e=e[nb:], phir=phir, ur=ur,
                                        npw=npw))
        self.dim = sum(b["phi"].shape[1] * nb for b in self.blocks)
        # basis bookkeeping
        self.offsets = []
        o = 0
        for b in self.blocks:
            self.offsets.append(o)
            o += nb * b["phi"].shape[1]
        # D and tau
        dvals = []
        jvals = []
        tau = np.zeros((self.dim, 4, nr), dtype=np.complex128)
        for bi, b in enumerate(self.blocks):
            t = np.ones(4) if b["side"] == 0 else np.array([1.0, -1.0, -1.0, -1.0])
            eocc = gs.evals[b["side"], b["k"]]
            nemp = b["phi"].shape[1]
            for n in range(nb):
                for c in range(nemp):
                    a = self.offsets[bi] + n * nemp + c
                    dvals.append(b["e"][c] - eocc[n])
                    jvals.append(1.0 if b["side"] == 0 else -1.0)
                    for al in range(4):
                        tau[a, al] = t[al] * np.einsum("sr,st,tr->r", b["ur"][n].conj(), SIG4[al],
                                                       b["phir"][:, :, c])
        self.D = np.array(dvals)
        self.J = np.array(jvals)
        # F tau
        ftau = np.zeros_like(tau)
        if gs.kernel_mask & 2:
            f = xc_matrix_from_table(fxc_table)
            ftau += np.einsum("abr,xbr->xar", f, tau)
        if gs.kernel_mask & 1:
            bvec = 2 * np.pi * np.linalg.inv(gs.lattice).T
            mg = _centered_millers(fft)
            qg = gs.q[None, :] + mg @ bvec
            qg2 = np.sum(qg * qg, axis=1)
            fac = np.where(0.5 * qg2 <= 4.0 * gs.ecutwfc, 4 * np.pi / qg2, 0.0)
            e = dft_matrix(mg, fft)  # (Nr, NG)
            vh = e @ (fac[:, None] * (e.conj().T @ tau[:, 0, :].T)) / nr
            ftau[:, 0, :] += vh.T
        w = gs.wk[0]
        assert np.allclose(gs.wk, w)
        self.K = w * (omega / nr) * (tau.reshape(self.dim, -1).conj() @ ftau.reshape(self.dim, -1).T)
        self.L = self.J[:, None] * (np.diag(self.D) + self.K)

    def to_br(self, a):
        gs = self.gs
        x = np.zeros(gs.br_shape, dtype=np.complex128)
        for bi, b in enumerate(self.blocks):
            nemp = b["phi"].shape[1]
            for n in range(gs.nocc):
                coef = a[self.offsets[bi] + n * nemp:self.offsets[bi] + (n + 1) * nemp]
                vec = b["phi"] @ coef
                x[b["side"], b["k"], n, 0, :b["npw"]] = vec[:b["npw"]]
                x[b["side"], b["k"], n, 1, :b["npw"]] = vec[b["npw"]:]
        return x

    def from_br(self, x):
        gs = self.gs
        a = np.zeros(self.dim, dtype=np.complex128)
        resid = 0.0
        for bi, b in enumerate(self.blocks):
            nemp = b["phi"].shape[1]
            for n in range(gs.nocc):
                vec = np.concatenate([x[b["side"], b["k"], n, 0, :b["npw"]],
                                      x[b["side"], b["k"], n, 1, :b["npw"]]])
                coef = b["phi"].conj().T @ vec
                a[self.offsets[bi] + n * nemp:self.offsets[bi] + (n + 1) * nemp] = coef
                resid = max(resid, np.linalg.norm(vec - b["phi"] @ coef))
        return a, resid

"""Model Hamiltonian H^(s)_p of Eq. H0_k_plus_q and its diagonalisation.

H^(s)_p = |p+G|^2/2 + v_loc + s B(r).sigma + V_NL,p,   s = +1 (X side), -1 (Y side)

Two routes, both on the same discrete operator:
* ``dense_hamiltonian``: explicit (2 Np x 2 Np) matrix from the grid Fourier
  coefficients of v_loc and B (circular convolution) plus the projector sum.
* ``HamiltonianFFT``: matrix-free application with FFTs (torch; CPU or CUDA),
  used by the iterative eigensolver for the larger bundles.
"""

from __future__ import annotations

import numpy as np
import scipy.fft

from .model import PAULI, miller_to_index


def grid_fourier(f_r: np.ndarray, fft) -> np.ndarray:
    """F[m] = (1/Nr) sum_j f(r_j) exp(-i G_m.r_j) on the grid (C order, flat)."""
    return scipy.fft.fftn(np.asarray(f_r).reshape(fft), workers=-1).ravel() / np.prod(fft)


def dense_hamiltonian(sign: int, p: np.ndarray, miller: np.ndarray, bvec: np.ndarray,
                      fft, vloc: np.ndarray, bfield: np.ndarray, beta: np.ndarray,
                      dnl: np.ndarray) -> np.ndarray:
    n1, n2, n3 = fft
    npw = miller.shape[0]
    dm = miller[:, None, :].astype(np.int64) - miller[None, :, :].astype(np.int64)
    idx = ((dm[..., 0] % n1) * n2 + (dm[..., 1] % n2)) * n3 + (dm[..., 2] % n3)
    vq = grid_fourier(vloc, fft)[idx]
    bq = [grid_fourier(bfield[i], fft)[idx] for i in range(3)]
    h = np.zeros((2 * npw, 2 * npw), dtype=np.complex128)
    for s in range(2):
        h[s * npw:(s + 1) * npw, s * npw:(s + 1) * npw] += vq
    for i in range(3):
        for s in range(2):
            for t in range(2):
                if PAULI[i, s, t] != 0:
                    h[s * npw:(s + 1) * npw, t * npw:(t + 1) * npw] += sign * PAULI[i, s, t] * bq[i]
    kin = 0.5 * np.sum((p[None, :] + miller @ bvec) ** 2, axis=1)
    h[np.arange(2 * npw), np.arange(2 * npw)] += np.concatenate([kin, kin])
    # V_NL = sum beta_i D_(i s),(j t) beta_j^H
    nproj = beta.shape[0]
    for s in range(2):
        for t in range(2):
            dst = dnl[s::2, t::2]  # (nproj, nproj)
            h[s * npw:(s + 1) * npw, t * npw:(t + 1) * npw] += beta.T @ dst @ beta.conj()
    assert nproj == dnl.shape[0] // 2
    return 0.5 * (h + h.conj().T)


class HamiltonianFFT:
    """Matrix-free H^(s)_p on spinor blocks X of shape (m, 2, Np) (torch)."""

    def __init__(self, torch, device, sign, p, miller, bvec, fft, vloc, bfield, beta, dnl):
        self.t = torch
        self.dev = device
        self.fft = tuple(fft)
        self.nr = int(np.prod(fft))
        self.npw = miller.shape[0]
        c = torch.complex128
        self.idx = torch.as_tensor(miller_to_index(miller, fft), device=device)
        self.kin = torch.as_tensor(0.5 * np.sum((p[None, :] + miller @ bvec) ** 2, axis=1),
                                   device=device)
        vr = torch.as_tensor(np.asarray(vloc).reshape(fft), device=device)
        b = [torch.as_tensor(np.asarray(bfield[i]).reshape(fft), device=device) for i in range(3)]
        # 2x2 local potential matrix on the grid: v + s B.sigma
        self.w00 = (vr + sign * b[2]).to(c)
        self.w11 = (vr - sign * b[2]).to(c)
        self.w01 = (sign * (b[0] - 1j * b[1])).to(c)
        self.w10 = (sign * (b[0] + 1j * b[1])).to(c)
        self.beta = torch.as_tensor(beta, device=device)
        self.dnl = torch.as_tensor(dnl, device=device)

    def __call__(self, x):
        t = self.t
        m = x.shape[0]
        grid = t.zeros((m, 2, self.nr), dtype=x.dtype, device=self.dev)
        grid[:, :, self.idx] = x
        psi = t.fft.ifftn(grid.reshape(m, 2, *self.fft), dim=(2, 3, 4))
        out0 = self.w00 * psi[:, 0] + self.w01 * psi[:, 1]
        out1 = self.w10 * psi[:, 0] + self.w11 * psi[:, 1]
        out = t.stack([out0, out1], dim=1)
        hg = t.fft.fftn(out, dim=(2, 3, 4)).reshape(m, 2, self.nr)[:, :, self.idx]
        hg = hg + self.kin * x
        proj = t.einsum("ig,msg->mis", self.beta.conj(), x).reshape(m, -1)  # (m, 2*nproj) idx 2i+s
        d = proj @ self.dnl.T
        d = d.reshape(m, -1, 2)
        hg = hg + t.einsum("ig,mis->msg", self.beta, d)
        return hg

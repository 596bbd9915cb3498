"""The Liouvillian in the batch representation (oracle; FP64, matrix-free).

A response vector x = (X, Y) holds, for every k point and occupied band n, the
spinor x_{n,k+q} (side X) and y_{n,k+q} (side Y) on the k+q plane-wave sphere
(Eq. batch_rho).  Layout: (2, nk, nocc, 2, npwx) complex128, zero padding.

L acts as (Eq. Liouvillian_BR_q and the block actions after it)

    out_X =  P_{k+q}  [ (H+_{k+q} - e_{n,k}) x_n + V'_HXC[x, y] U_{n,k} ]
    out_Y = -P+_{k+q} [ (H-_{k+q} - e_{n,k}) y_n + V'+_HXC[x, y] (T U)_{n,k} ]

with H+- of Eq. H0_k_plus_q (exchange field +-B), V'_HXC of Eq. V_HXC_resp_q
built from the response densities of Eqs. charge_dens_resp_q / spin_dens_resp_q
(the Y side enters the magnetisation with a minus sign), V'+ = V' with the
magnetic part reversed, and P, P+ the empty-manifold projectors of Eqs.
P_minus_q2 / P_plus_q2 built from the occupied k+q states.  P is applied to the
whole row (reading: equal to the paper's placement in exact arithmetic).
"""

from __future__ import annotations

import numpy as np

from . import grid, xc

PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)
SIGMA4 = np.concatenate([np.eye(2, dtype=np.complex128)[None], PAULI], axis=0)  # sigma_0..3
T_SIGN = np.array([1.0, -1.0, -1.0, -1.0])  # Y-side sign per density component


def component(mu):
    """(sigma, Y-side sign t) of perturbation / observable index mu: 0, 1, 2 = the spin
    components x, y, z (Eq. spin_dens_resp_q, t = -1) and 3 = the charge (sigma^0,
    Eq. charge_dens_resp_q, t = +1) of the 4x4 generalised susceptibility."""
    a = 0 if mu == 3 else mu + 1
    return SIGMA4[a], T_SIGN[a]


def reciprocal(lattice):
    return 2.0 * np.pi * np.linalg.inv(lattice).T


class Liouvillian:
    def __init__(self, gs):
        self.gs = gs
        self.fft = tuple(gs.fft)
        self.nr = int(np.prod(self.fft))
        self.omega = float(abs(np.linalg.det(gs.lattice)))
        self.bvec = reciprocal(gs.lattice)
        self.idx_k, self.idx_kq, self.kin = [], [], []
        for k in range(gs.nk):
            mk = gs.miller_k[k, :gs.npw_k[k]]
            mkq = gs.miller_kq[k, :gs.npw_kq[k]]
            self.idx_k.append(grid.flat_index(mk, self.fft))
            self.idx_kq.append(grid.flat_index(mkq, self.fft))
            kqg = gs.kpts[k] + gs.q + mkq @ self.bvec
            self.kin.append(0.5 * np.sum(kqg * kqg, axis=1))
        # Hartree factor 4 pi / |q+G|^2 on the density sphere |q+G|^2/2 <= 4 ecutwfc
        qg = gs.q[None, :] + grid.grid_millers(self.fft) @ self.bvec
        qg2 = np.sum(qg * qg, axis=1)
        self.vh_fac = np.where(0.5 * qg2 <= 4.0 * gs.ecutwfc, 4.0 * np.pi / qg2, 0.0)
        self.fxc = xc.kernel_table(gs.n0, gs.m0)
        # local 2x2 ground-state potential per side: v_loc + s B.sigma
        self.vloc = gs.vloc
        self.bfield = gs.bfield

    # ----------------------------------------------------------------- helpers
    def u_real(self, side, k):
        """Real-space occupied orbitals U^side_{n,k}(r): (nocc, 2, Nr)."""
        gs = self.gs
        c = gs.coeff_k[side, k, :, :, :gs.npw_k[k]]
        return grid.sphere_to_real(c, self.idx_k[k], self.fft, self.omega)

    def x_real(self, x, side, k):
        c = x[side, k, :, :, :self.gs.npw_kq[k]]
        return grid.sphere_to_real(c, self.idx_kq[k], self.fft, self.omega)

    def response_density(self, x):
        """rho'_a(r), a = 0..3 (Eqs. charge_dens_resp_q, spin_dens_resp_q)."""
        gs = self.gs
        rho = np.zeros((4, self.nr), dtype=np.complex128)
        for side in range(2):
            for k in range(gs.nk):
                u = self.u_real(side, k)
                xr = self.x_real(x, side, k)
                for a in range(4):
                    t = 1.0 if side == 0 else T_SIGN[a]
                    # sum_n U_n^dagger sigma_a x_n
                    val = np.einsum("nsr,st,ntr->r", u.conj(), SIGMA4[a], xr)
                    rho[a] += gs.wk[k] * t * val
        return rho

    def hxc_potential(self, rho):
        """v'_a(r) = delta_a0 v'_H + sum_b f_ab rho'_b (Eqs. v_H_q, v_XC_q, b_XC_q)."""
        v = np.zeros_like(rho)
        if self.gs.kernel_mask & 1:
            rg = grid.fftn(rho[0].reshape(self.fft)).ravel() / self.nr
            vh = grid.ifftn((self.vh_fac * rg).reshape(self.fft)).ravel() * self.nr
            v[0] += vh
        if self.gs.kernel_mask & 2:
            v += xc.apply_kernel(self.fxc, rho)
        return v

    def project_empty(self, h, side, k):
        """h <- h - sum_m U_m <U_m|h> over occupied k+q states (Eqs. P_minus_q2, P_plus_q2)."""
        gs = self.gs
        npw = gs.npw_kq[k]
        u = gs.coeff_kq[side, k, :, :, :npw].reshape(gs.nocc, -1)
        hv = h.reshape(h.shape[0], -1)
        s = u.conj() @ hv.T  # (m, n) = <U_m | h_n>
        return (hv - (u.T @ s).T).reshape(h.shape)

    def nonlocal_apply(self, xs, k):
        """V_NL x = sum_ij beta_i D_(i s)(j t) <beta_j | x_t>; xs: (n, 2, npw)."""
        gs = self.gs
        npw = gs.npw_kq[k]
        beta = gs.beta_kq[k, :, :npw]
        proj = np.einsum("ig,nsg->nis", beta.conj(), xs)  # (n, nproj, 2)
        d = np.einsum("ab,nb->na", gs.dnl, proj.reshape(xs.shape[0], -1)).reshape(proj.shape)
        return np.einsum("ig,nis->nsg", beta, d)

    # ------------------------------------------------------------------ apply
    def apply(self, x, kpoints=None):
        """L x.  kpoints (optional): compute the output only at these k points and leave
        the rest zero; the response density still sums over every k point."""
        gs = self.gs
        x = np.asarray(x, dtype=np.complex128)
        kset = range(gs.nk) if kpoints is None else sorted(set(int(k) for k in kpoints))
        rho = self.response_density(x)
        v = self.hxc_potential(rho)
        out = np.zeros_like(x)
        for side in range(2):
            s = 1.0 if side == 0 else -1.0
            # W^X = v0 + v.sigma ; W^Y = v0 - v.sigma (V'+ reverses the magnetic part)
            w = SIGMA4[0][:, :, None] * v[0][None, None, :]
            for i in range(3):
                w = w + s * PAULI[i][:, :, None] * v[1 + i][None, None, :]
            # ground local potential v_loc + s B.sigma
            h0 = SIGMA4[0][:, :, None] * self.vloc[None, None, :]
            for i in range(3):
                h0 = h0 + s * PAULI[i][:, :, None] * self.bfield[i][None, None, :]
            for k in kset:
                npw = gs.npw_kq[k]
                xs = x[side, k, :, :, :npw]
                u = self.u_real(side, k)
                xr = self.x_real(x, side, k)
                prod = np.einsum("str,ntr->nsr", h0, xr) + np.einsum("str,ntr->nsr", w, u)
                h = grid.real_to_sphere(prod, self.idx_kq[k], self.fft, self.omega)
                h += self.kin[k][None, None, :] * xs
                h += self.nonlocal_apply(xs, k)
                h -= gs.evals[side, k][:, None, None] * xs
                h = self.project_empty(h, side, k)
                out[side, k, :, :, :npw] = h if side == 0 else -h
        return out

    def apply_adjoint(self, x):
        """L^H = J L J (pseudo-Hermiticity with J = diag(+1 on X, -1 on Y))."""
        return jmul(self.apply(jmul(x)))

    # ------------------------------------------------------------ end vectors
    def sigma_u_on_kq(self, mu):
        """(2, nk, nocc, 2, npwx): sigma^mu U^side_{n,k} expressed on the k+q sphere
        (mu = 3: sigma^0, the charge)."""
        gs = self.gs
        sig = component(mu)[0]
        out = np.zeros(gs.br_shape, dtype=np.complex128)
        for side in range(2):
            for k in range(gs.nk):
                box = np.zeros((gs.nocc, 2, self.nr), dtype=np.complex128)
                box[:, :, self.idx_k[k]] = gs.coeff_k[side, k, :, :, :gs.npw_k[k]]
                cq = box[:, :, self.idx_kq[k]]
                out[side, k, :, :, :gs.npw_kq[k]] = np.einsum("st,ntg->nsg", sig, cq)
        return out

    def start_vector(self, mu):
        """v^mu = P J u^mu = (P sigma^mu U, -t P+ sigma^mu T U)  (Sec. 2.5; the
        commutator with the ground state puts J on the perturbation's BR image): for the
        spin components (P sigma U, P+ sigma T U), for the charge (P U, -P+ T U)."""
        gs = self.gs
        su = self.sigma_u_on_kq(mu)
        su[1] *= -component(mu)[1]
        for side in range(2):
            for k in range(gs.nk):
                npw = gs.npw_kq[k]
                su[side, k, :, :, :npw] = self.project_empty(su[side, k, :, :, :npw], side, k)
        return su

    def left_vector(self, lam):
        """u^lambda = (sigma^lambda U, t sigma^lambda T U): the vector whose scalar product
        with a BR vector is its response density lambda (Eqs. charge_dens_resp_q,
        spin_dens_resp_q: t = +1 for the charge, -1 for the spin components)."""
        u = self.sigma_u_on_kq(lam)
        u[1] *= component(lam)[1]
        return u


def jmul(x):
    y = np.array(x, dtype=np.complex128, copy=True)
    y[1] *= -1.0
    return y


def jdot(a, b):
    """a^H J b."""
    return np.vdot(a[0], b[0]) - np.vdot(a[1], b[1])

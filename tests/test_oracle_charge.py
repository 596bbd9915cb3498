"""The charge column and row of the 4x4 generalised susceptibility (oracle, CPU).

The paper's formalism gives the whole 4x4 matrix chi_{lambda mu}, lambda, mu in {x, y, z,
charge}: the charge perturbation and observable use sigma^0 where the spin ones use the
Pauli matrices, and the Y side of the response density enters the charge with + and the
magnetisation with - (Eqs. charge_dens_resp_q, spin_dens_resp_q).  Index 3 is the charge.

Pins:
* u^lambda . x is the q component of the response density lambda of x (the oracle's
  response density, itself pinned against the brute-force particle-hole L): the same
  ratio Omega / (N_r w) for the charge and the three spin components;
* with the kernel off, all 16 components from NH chains equal the sum over transitions
  chi0_{lm} = w sum [conj(M^l_X) M^m_X / (w + i eta - D_X)
                     - t_l t_m conj(M^l_Y) M^m_Y / (w + i eta + D_Y)],
  M = <c|sigma|n> from the dense diagonalisation and t the time-reversal parity of the
  operator (+1 charge, -1 spin);
* with the kernel on, the 4x4 chi of the chains equals the direct resolvent of the
  brute-force L, and the static charge response chi_00(q, 0) is real and negative;
* collinear case without spin-orbit coupling: the charge does not couple to the
  transverse spin components (chi_0x = chi_x0 = chi_0y = chi_y0 = 0).
"""

import numpy as np
import pytest

from _cases import liouvillian, particle_hole
from oracle.lanczos import run_chain
from oracle.liouvillian import component
from oracle.spectrum import HA_MEV, chi_thomas

OMEGAS = np.linspace(0.0, 0.3, 31)
T_PARITY = {0: -1.0, 1: -1.0, 2: -1.0, 3: 1.0}


def test_left_vectors_give_the_response_density():
    lv = liouvillian("C0K")
    gs = lv.gs
    rng = np.random.default_rng(5)
    x = rng.standard_normal(gs.br_shape) + 1j * rng.standard_normal(gs.br_shape)
    for k in range(gs.nk):
        x[:, k, :, :, gs.npw_kq[k]:] = 0
    rho = lv.response_density(x)  # components 0..3 = charge, x, y, z
    w = gs.wk[0]
    for lam in range(4):
        a = 0 if lam == 3 else lam + 1
        ref = gs.omega / (lv.nr * w) * np.sum(rho[a])
        got = np.vdot(lv.left_vector(lam), x)
        assert abs(got - ref) <= 1e-12 * abs(ref), (lam, got, ref)


def _transitions(ph, lv):
    """Per block: the empty-state energies, occupied energies and <c|sigma^m|n> for the
    four components m (explicit matrix elements of the dense diagonalisation)."""
    gs = lv.gs
    out = []
    for b in ph.blocks:
        side, k = b["side"], b["k"]
        npw = b["npw"]
        mats = []
        for m in range(4):
            su = lv.sigma_u_on_kq(m)[side, k, :, :, :npw]  # (nocc, 2, npw): sigma^m U
            vec = np.concatenate([su[:, 0], su[:, 1]], axis=1)  # (nocc, 2 npw)
            mats.append(b["phi"].conj().T @ vec.T)  # (nemp, nocc)
        out.append((side, b["e"], gs.evals[side, k], mats))
    return out


def test_chi0_sum_over_transitions_all_components():
    lv, ph = liouvillian("C0", 0), particle_hole("C0", 0)
    w = lv.gs.wk[0]
    eta = 10.0 / HA_MEV
    tr = _transitions(ph, lv)
    ref = np.zeros((4, 4, len(OMEGAS)), dtype=np.complex128)  # [mu][lam][omega]
    for side, e_emp, e_occ, mats in tr:
        d = e_emp[:, None] - e_occ[None, :]
        for mu in range(4):
            for lam in range(4):
                num = np.conj(mats[lam]) * mats[mu]
                for i, om in enumerate(OMEGAS):
                    if side == 0:
                        ref[mu, lam, i] += w * np.sum(num / (om + 1j * eta - d))
                    else:
                        ref[mu, lam, i] -= (T_PARITY[lam] * T_PARITY[mu] * w
                                            * np.sum(num / (om + 1j * eta + d)))
    scale = np.abs(ref).max()
    for mu in range(4):
        got = chi_thomas(run_chain(lv, mu, 700, "nh", ncomp=4), OMEGAS, eta, w)
        assert np.abs(got - ref[mu]).max() <= 1e-8 * scale, mu


def _direct4(ph, lv, omegas, eta):
    va = [ph.from_br(lv.start_vector(m))[0] for m in range(4)]
    ua = [ph.from_br(lv.left_vector(l))[0] for l in range(4)]
    w = lv.gs.wk[0]
    out = np.zeros((4, 4, len(omegas)), dtype=np.complex128)
    for i, om in enumerate(omegas):
        y = np.linalg.solve((om + 1j * eta) * np.eye(ph.dim) - ph.L, np.stack(va, axis=1))
        for m in range(4):
            for l in range(4):
                out[m, l, i] = w * np.vdot(ua[l], y[:, m])
    return out


def test_chi_4x4_with_kernel_and_static_charge_response():
    lv, ph = liouvillian("C0"), particle_hole("C0")
    eta = 10.0 / HA_MEV
    ref = _direct4(ph, lv, OMEGAS, eta)
    w = lv.gs.wk[0]
    for mu in range(4):
        got = chi_thomas(run_chain(lv, mu, 800, "nh", ncomp=4), OMEGAS, eta, w)
        assert np.linalg.norm(got - ref[mu]) <= 1e-7 * np.linalg.norm(ref[mu][mu]), mu
    # static density-density response of a stable system: real and negative
    st = _direct4(ph, lv, [0.0], 1e-9)[3, 3, 0]
    assert st.real < 0 and abs(st.imag) <= 1e-6 * abs(st.real), st


def test_collinear_charge_decouples_from_transverse_spin():
    lv = liouvillian("C0", 3, True)
    eta = 0.05
    chi = np.array([chi_thomas(run_chain(lv, mu, 300, "nh", ncomp=4), OMEGAS, eta,
                               lv.gs.wk[0]) for mu in range(4)])  # chi[mu][lam]
    scale = np.abs(chi).max()
    for a, b in ((3, 0), (0, 3), (3, 1), (1, 3)):
        assert np.abs(chi[a][b]).max() <= 1e-12 * scale, (a, b)
    assert np.abs(chi[3][2]).max() >= 1e-6 * scale  # charge and longitudinal spin couple
    assert np.abs(chi[3][3]).max() >= 1e-3 * scale


def test_component_convention():
    assert np.allclose(component(3)[0], np.eye(2)) and component(3)[1] == 1.0
    for mu in range(3):
        assert component(mu)[1] == -1.0

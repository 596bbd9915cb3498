"""Pins of the oracle's matrix-free Liouvillian (CPU only).

P1: against the brute-force particle-hole matrix L = J (D + K) assembled from a
full diagonalisation of explicit dense Hamiltonians (tests/_bruteforce.py), for
every kernel mask (independent particles, Hartree only, XC only, both) and for
one and two k points.  P2: the pseudo-Hermiticity x^H J L y = (L x)^H J y on
range(P_c) (Sec. 2.5: the property the pseudo-Hermitian recursion relies on).
Plus: L^H = J L J against the dense adjoint; the start vector lies in range(P_c);
the output of L always lies in range(P_c) (Eqs. P_minus_q2 / P_plus_q2).
"""

import numpy as np
import pytest

from _cases import liouvillian, particle_hole
from oracle.liouvillian import jdot


@pytest.mark.parametrize("name", ["C0", "C0K"])
@pytest.mark.parametrize("mask", [0, 1, 2, 3])
def test_matrix_free_equals_bruteforce(name, mask):
    lv = liouvillian(name, mask)
    ph = particle_hole(name, mask)
    rng = np.random.default_rng(3 + mask)
    a = rng.standard_normal(ph.dim) + 1j * rng.standard_normal(ph.dim)
    y = lv.apply(ph.to_br(a))
    b, outside = ph.from_br(y)
    ref = ph.L @ a
    assert np.linalg.norm(b - ref) <= 1e-12 * np.linalg.norm(ref)
    assert outside <= 1e-12 * np.linalg.norm(y)


def test_apply_restricted_to_sampled_k_points():
    """Outputs at a subset of k points (the density still over every k) equal the
    brute-force L at those k points; the other k points stay zero."""
    lv = liouvillian("C0K")
    ph = particle_hole("C0K")
    assert lv.gs.nk >= 2
    rng = np.random.default_rng(17)
    a = rng.standard_normal(ph.dim) + 1j * rng.standard_normal(ph.dim)
    ref = ph.to_br(ph.L @ a)
    ks = [lv.gs.nk - 1]
    y = lv.apply(ph.to_br(a), kpoints=ks)
    assert np.linalg.norm(y[:, ks] - ref[:, ks]) <= 1e-12 * np.linalg.norm(ref[:, ks])
    rest = [k for k in range(lv.gs.nk) if k not in ks]
    assert not y[:, rest].any()


@pytest.mark.parametrize("name", ["C0", "C0K"])
def test_adjoint_is_jlj(name):
    lv = liouvillian(name)
    ph = particle_hole(name)
    rng = np.random.default_rng(9)
    a = rng.standard_normal(ph.dim) + 1j * rng.standard_normal(ph.dim)
    b, _ = ph.from_br(lv.apply_adjoint(ph.to_br(a)))
    ref = ph.L.conj().T @ a
    assert np.linalg.norm(b - ref) <= 1e-12 * np.linalg.norm(ref)


def test_pseudo_hermiticity_on_range_pc():
    lv = liouvillian("C0K")
    ph = particle_hole("C0K")
    rng = np.random.default_rng(21)
    x = ph.to_br(rng.standard_normal(ph.dim) + 1j * rng.standard_normal(ph.dim))
    y = ph.to_br(rng.standard_normal(ph.dim) + 1j * rng.standard_normal(ph.dim))
    lhs = jdot(x, lv.apply(y))
    rhs = jdot(lv.apply(x), y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # and the Hermitian part D + K is positive for the full kernel on this model
    h = np.diag(ph.D) + ph.K
    assert np.allclose(h, h.conj().T, atol=1e-13 * np.abs(h).max())
    assert np.linalg.eigvalsh(h).min() > 0


@pytest.mark.parametrize("mu", [0, 1, 2])
def test_start_vector_in_range_pc(mu):
    lv = liouvillian("C0K")
    ph = particle_hole("C0K")
    v = lv.start_vector(mu)
    _, outside = ph.from_br(v)
    assert outside <= 1e-12 * np.linalg.norm(v)
    # u^lambda = J sigma U: its X block equals the unprojected sigma U on the k+q sphere
    u = lv.left_vector(mu)
    su = lv.sigma_u_on_kq(mu)
    assert np.array_equal(u[0], su[0]) and np.array_equal(u[1], -su[1])


def test_independent_particle_eigenvalues():
    """With the kernel off, L = J D: its spectrum is +-(e_c(k+q) - e_n(k))."""
    ph = particle_hole("C0", 0)
    ev = np.sort(np.linalg.eigvals(ph.L).real)
    ref = np.sort(ph.J * ph.D)
    assert np.max(np.abs(ev - ref)) < 1e-11


def _larmor_case(self_consistent):
    from synth import make_ground_state
    kw = dict(collinear=True, kernel_mask=2, q_2pi_a=(1e-4, 0.0, 0.0))
    if self_consistent:
        kw.update(self_consistent=True, b_ext=0.05)
    return make_ground_state("C0", **kw)


def test_larmor_mode_of_self_consistent_model():
    """Physical pin of the transverse ALSDA kernel, the response densities and the
    potential coupling: in a self-consistent collinear model without spin-orbit
    coupling, with a uniform external field b_ext along z on top of the exchange
    field of its own magnetisation, the uniform spin precession is an eigenmode of
    L at exactly 2 b_ext (Larmor theorem; here at q -> 0, |q| = 1e-4 2pi/a).  The
    same crystal with a fixed, non-self-consistent field has no such mode at 2|B|."""
    from oracle.liouvillian import Liouvillian
    from _bruteforce import ParticleHole
    gs = _larmor_case(True)
    lv = Liouvillian(gs)
    ph = ParticleHole(gs, lv.fxc)
    ev, vec = np.linalg.eig(ph.L)
    i = int(np.argmin(np.abs(ev - 0.1)))
    assert abs(ev[i] - 0.1) <= 1e-7, ev[i]
    # the oracle's matrix-free L reproduces the eigenpair
    x = ph.to_br(vec[:, i])
    y = lv.apply(x)
    assert np.linalg.norm(y - 0.1 * x) <= 1e-7 * np.linalg.norm(x)
    gs2 = _larmor_case(False)
    lv2 = Liouvillian(gs2)
    ev2 = np.linalg.eigvals(ParticleHole(gs2, lv2.fxc).L)
    assert np.min(np.abs(ev2 - 2 * 0.2)) > 1e-3

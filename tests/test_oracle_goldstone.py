"""Goldstone check of the oracle's Liouvillian on a spontaneously magnetic model.

The paper's dispersion discussion: without spin-orbit coupling the lowest magnon of a
ferromagnet goes to zero energy as q -> 0 (the rotational symmetry of the spin space is
broken spontaneously), and spin-orbit coupling opens a gap there.

Model ("CG" in synth.configs): two electrons per simple-cubic cell (a = 8 bohr) bound
in two deep Gaussian wells 3.5 bohr apart.  The self-consistent Slater exchange (no
external field) polarises both electrons in parallel (|M| = 2).  The cutoff lies halfway
between two shells of |G|^2, so the k+q sphere equals the k sphere for the q used here
and L changes smoothly with q.  The spin-orbit term lambda L_z sigma_z / 2 (lambda =
0.9 Ha) sits on p projectors 0.7 bohr off the first well.

Checks on the brute-force particle-hole L (tests/_bruteforce.py, full diagonalisation):
* without spin-orbit coupling the lowest pair of eigenvalues is +-omega(q), real, with
  omega(2q) = 4 omega(q) (quadratic dispersion) and omega -> 0 when fitted to a + b q^2;
  the oracle's matrix-free L reproduces that eigenpair;
* with spin-orbit coupling the pair stays at +-(Delta + O(q)) with Delta = 5.2e-4 Ha
  (14 meV) extrapolated to q = 0 from either branch.
A single electron per cell would not do: any superposition of its Kramers pair keeps
|m(r)| = n(r) at every point, so the LSDA energy does not depend on the direction of
the moment and the zero mode survives spin-orbit coupling.
"""

import functools

import numpy as np
import pytest

from synth import make_ground_state

QS = (0.005, 0.01, 0.02)


@functools.lru_cache(maxsize=None)
def case(soc: bool, q: float):
    from oracle.liouvillian import Liouvillian
    from _bruteforce import ParticleHole
    gs = make_ground_state("CG", collinear=not soc, self_consistent=True, b_ext=0.0,
                           q_2pi_a=(q, 0.0, 0.0))
    lv = Liouvillian(gs)
    ph = ParticleHole(gs, lv.fxc)
    ev, vec = np.linalg.eig(ph.L)
    order = np.argsort(np.abs(ev))[:2]
    order = order[np.argsort(ev[order].real)]  # (negative, positive)
    return gs, lv, ph, ev[order], vec[:, order], np.sort(np.abs(ev))[2]


def test_spontaneous_magnetisation():
    gs = case(False, QS[1])[0]
    mtot = gs.m0.mean(axis=1) * gs.omega
    assert abs(abs(mtot[2]) - 2.0) <= 1e-6 and np.hypot(mtot[0], mtot[1]) <= 1e-9, mtot
    assert gs.meta["gap_min"] >= 1e-3


def test_goldstone_mode_without_spin_orbit():
    om = []
    for q in QS:
        _, _, _, pair, _, nxt = case(False, q)
        assert np.max(np.abs(pair.imag)) <= 1e-12
        assert abs(pair[0].real + pair[1].real) <= 1e-10, pair  # +-omega
        assert nxt >= 0.1  # the pair is isolated
        om.append(pair[1].real)
    om = np.array(om)
    assert np.all(om > 0)
    ratio = om[1:] / om[:-1]
    assert np.all(np.abs(ratio - 4.0) <= 0.02), ratio  # quadratic in q
    a, b = np.polyfit(np.array(QS) ** 2, om, 1)[::-1]
    assert abs(a) <= 1e-9, (a, b)  # omega -> 0 as q -> 0
    # the matrix-free L of the oracle maps the eigenvector to omega times itself
    gs, lv, ph, pair, vec, _ = case(False, QS[1])
    x = ph.to_br(vec[:, 1])
    assert np.linalg.norm(lv.apply(x) - pair[1] * x) <= 1e-10 * np.linalg.norm(x)


def test_spin_orbit_opens_a_gap():
    pos, neg = [], []
    for q in QS[:2]:
        _, _, _, pair, _, nxt = case(True, q)
        assert np.max(np.abs(pair.imag)) <= 1e-12 and nxt >= 0.1
        neg.append(pair[0].real)
        pos.append(pair[1].real)
    # extrapolate each branch linearly to q = 0 (the O(q) part is the nonreciprocal shift)
    d_pos = 2 * pos[0] - pos[1]
    d_neg = -(2 * neg[0] - neg[1])
    assert abs(d_pos - d_neg) <= 1e-6, (d_pos, d_neg)
    assert 4e-4 <= d_pos <= 7e-4, d_pos
    # and far above the spin-orbit-free mode at the same q
    assert min(pos) >= 100 * case(False, QS[1])[3][1].real

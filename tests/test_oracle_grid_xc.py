"""Pins of the oracle's grid maps, Hartree term and XC kernel (CPU only).

* sphere <-> grid maps and the Hartree potential against explicit DFT /
  Coulomb sums on an 8^3 grid (the library FFT is not trusted here);
* the LSDA kernel table against central finite differences of the exchange
  energy density e_x(n, m) it is derived from (Eqs. v_XC_q, b_XC_q);
* its |m| -> 0 limit (isotropic, f_0i = 0) and low-density cutoff.
"""

import numpy as np
import pytest

from oracle import grid, xc


def _random_sphere(rng, fft, n):
    ax = [np.arange(-(m // 2) + 1, (m - 1) // 2) for m in fft]
    all_m = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    sel = rng.choice(all_m.shape[0], size=n, replace=False)
    return all_m[sel]


def test_sphere_to_real_matches_direct_sum():
    rng = np.random.default_rng(11)
    fft = (8, 8, 8)
    omega = 123.4
    mil = _random_sphere(rng, fft, 40)
    c = rng.standard_normal((3, 40)) + 1j * rng.standard_normal((3, 40))
    got = grid.sphere_to_real(c, grid.flat_index(mil, fft), fft, omega)
    j = np.stack(np.meshgrid(*[np.arange(n) for n in fft], indexing="ij"), -1).reshape(-1, 3)
    ph = np.exp(2j * np.pi * (j / np.array(fft)) @ mil.T)  # (Nr, npw)
    ref = (ph @ c.T).T / np.sqrt(omega)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # forward map is the inverse on the sphere, and equals the explicit sum
    back = grid.real_to_sphere(ref, grid.flat_index(mil, fft), fft, omega)
    assert np.max(np.abs(back - c)) <= 1e-13 * np.max(np.abs(c))
    f = rng.standard_normal((2, 512)) + 1j * rng.standard_normal((2, 512))
    ref2 = (np.sqrt(omega) / 512) * (f @ ph.conj())
    got2 = grid.real_to_sphere(f, grid.flat_index(mil, fft), fft, omega)
    assert np.max(np.abs(got2 - ref2)) <= 1e-13 * np.max(np.abs(ref2))


def test_hartree_matches_coulomb_sum():
    """v_H(r) = sum_G 4 pi rho(G) / |q+G|^2 e^{iG.r} (Eq. v_H_q) by explicit sums."""
    from synth import make_ground_state
    from oracle.liouvillian import Liouvillian
    gs = make_ground_state("C0")
    gs = gs.__class__(**{**gs.__dict__, "kernel_mask": 1})
    lv = Liouvillian(gs)
    rng = np.random.default_rng(5)
    rho = np.zeros((4, gs.nr), dtype=np.complex128)
    rho[0] = rng.standard_normal(gs.nr) + 1j * rng.standard_normal(gs.nr)
    got = lv.hxc_potential(rho)[0]
    fft = gs.fft
    bvec = 2 * np.pi * np.linalg.inv(gs.lattice).T
    j = np.stack(np.meshgrid(*[np.arange(n) for n in fft], indexing="ij"), -1).reshape(-1, 3)
    mg = np.stack(np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in fft], indexing="ij"),
                  -1).reshape(-1, 3)
    ph = np.exp(2j * np.pi * (j / np.array(fft)) @ mg.T)
    rg = ph.conj().T @ rho[0] / gs.nr
    qg = gs.q[None, :] + mg @ bvec
    qg2 = np.sum(qg * qg, 1)
    fac = np.where(0.5 * qg2 <= 4 * gs.ecutwfc, 4 * np.pi / qg2, 0.0)
    ref = ph @ (fac * rg)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the q+G = q term is present (q != 0) and the sphere cut is active
    assert fac.max() == pytest.approx(4 * np.pi / np.dot(gs.q, gs.q))
    assert np.count_nonzero(fac == 0.0) > 0


@pytest.mark.parametrize("seed", range(6))
def test_kernel_matches_finite_differences(seed):
    rng = np.random.default_rng(100 + seed)
    n = rng.uniform(0.02, 0.3)
    m = rng.standard_normal(3)
    m *= rng.uniform(0.05, 0.8) * n / np.linalg.norm(m)
    f = xc.point_kernel(n, m)

    def e(rho):
        return xc.slater_energy(rho[0], np.linalg.norm(rho[1:]))

    rho0 = np.concatenate([[n], m])
    h = 1e-4 * n
    fd = np.zeros((4, 4))
    for a in range(4):
        for b in range(4):
            ea = np.eye(4)[a] * h
            eb = np.eye(4)[b] * h
            fd[a, b] = (e(rho0 + ea + eb) - e(rho0 + ea - eb) - e(rho0 - ea + eb)
                        + e(rho0 - ea - eb)) / (4 * h * h)
    assert np.max(np.abs(f - fd)) <= 1e-6 * np.max(np.abs(f))
    assert np.allclose(f, f.T)


def test_kernel_limits():
    n = 0.1
    f = xc.point_kernel(n, np.zeros(3))
    fs = -(1.0 / 3.0) * xc.C6PI * (0.5 * n) ** (-2.0 / 3.0)
    assert np.allclose(f, 0.5 * fs * np.eye(4), rtol=1e-14)
    # small |m| approaches the same isotropic limit continuously
    f2 = xc.point_kernel(n, np.array([0.0, 0.0, 1e-7]))
    assert np.max(np.abs(f2 - f)) < 1e-4 * np.abs(fs)
    assert not xc.point_kernel(1e-11, np.array([0.0, 0.0, 1e-12])).any()


def test_kernel_table_layout():
    rng = np.random.default_rng(3)
    n0 = rng.uniform(0.01, 0.2, 7)
    m0 = rng.standard_normal((3, 7)) * 0.01
    tab = xc.kernel_table(n0, m0)
    rho = rng.standard_normal((4, 7)) + 1j * rng.standard_normal((4, 7))
    v = xc.apply_kernel(tab, rho)
    for j in range(7):
        assert np.allclose(v[:, j], xc.point_kernel(n0[j], m0[:, j]) @ rho[:, j], rtol=1e-14)

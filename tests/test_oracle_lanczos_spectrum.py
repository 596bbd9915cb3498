"""Pins of the oracle's Lanczos recursions and spectrum (CPU only).

P3  closed-form independent-particle chi0 (kernel off) vs Lanczos + spectrum
P4  direct resolvent chi = w u^H (omega + i eta - L)^{-1} v by dense solves
P5  moments: w n0 sum_i conj(z_i) (T^k e1)_i = w u^H L^k v for k < 10
P6  non-Hermitian and pseudo-Hermitian chains give the same chi at convergence
P7  biorthogonality p_i^H q_j = delta_ij (NH, and PHM with p = J L q) and
    q_i^H J q_j = s_i delta_ij (PH, relative to ||q_i|| ||q_j||: the indefinite
    metric loses it quickly, which is recorded, not hidden)
P8  collinear special case ([H, S_z] = 0): chi_xz = chi_zx = 0, chi_xx = chi_yy,
    chi_xy = -chi_yx
P9  sum rule: int chi d omega = -i pi w u^H v (residue sum)
P12 Lanczos on the dense brute-force L equals the matrix-free chain step by step
Plus Thomas elimination vs pivoted banded LAPACK.
"""

import numpy as np
import pytest

from _cases import ground_state, liouvillian, particle_hole
from oracle.lanczos import lanczos_nh, lanczos_ph, lanczos_phm, run_chain
from oracle.liouvillian import jdot
from oracle.spectrum import HA_MEV, chi_banded, chi_thomas

OMEGAS = np.linspace(0.0, 0.3, 31)


def _direct(ph, lv, mu, omegas, eta):
    va, _ = ph.from_br(lv.start_vector(mu))
    ua = [ph.from_br(lv.left_vector(l))[0] for l in range(3)]
    w = lv.gs.wk[0]
    out = np.zeros((3, len(omegas)), dtype=np.complex128)
    for i, om in enumerate(omegas):
        y = np.linalg.solve((om + 1j * eta) * np.eye(ph.dim) - ph.L, va)
        for l in range(3):
            out[l, i] = w * np.vdot(ua[l], y)
    return out


@pytest.fixture(scope="module")
def c0_chains():
    lv = liouvillian("C0")
    return {f: [run_chain(lv, mu, 800 if f != "phm" else 600, f, keep_basis=20) for mu in range(3)]
            for f in ("nh", "ph", "phm")}


@pytest.mark.parametrize("flavor", ["nh", "phm"])
def test_p4_direct_resolvent(c0_chains, flavor):
    lv, ph = liouvillian("C0"), particle_hole("C0")
    eta = 10.0 / HA_MEV
    for mu in (0, 2):
        ref = _direct(ph, lv, mu, OMEGAS, eta)
        got = chi_thomas(c0_chains[flavor][mu], OMEGAS, eta, lv.gs.wk[0])
        assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref[mu])


def test_p6_nh_equals_ph(c0_chains):
    lv, ph = liouvillian("C0"), particle_hole("C0")
    eta = 0.1
    for mu in range(3):
        ref = _direct(ph, lv, mu, OMEGAS, eta)
        x_nh = chi_thomas(c0_chains["nh"][mu], OMEGAS, eta, lv.gs.wk[0])
        x_ph = chi_thomas(c0_chains["ph"][mu], OMEGAS, eta, lv.gs.wk[0])
        x_pm = chi_thomas(c0_chains["phm"][mu], OMEGAS, eta, lv.gs.wk[0])
        nrm = np.linalg.norm(ref[mu])
        assert np.linalg.norm(x_nh - ref) <= 1e-8 * nrm
        assert np.linalg.norm(x_ph - ref) <= 1e-8 * nrm
        assert np.linalg.norm(x_pm - ref) <= 1e-8 * nrm
        assert np.linalg.norm(x_ph - x_nh) <= 1e-8 * nrm


@pytest.mark.parametrize("flavor", ["nh", "ph", "phm"])
def test_p5_moments(c0_chains, flavor):
    lv = liouvillian("C0")
    w = lv.gs.wk[0]
    for mu in range(3):
        c = c0_chains[flavor][mu]
        m = 40
        t = np.diag(c.alpha[:m]) + np.diag(c.beta[:m - 1], -1) + np.diag(c.gamma[:m - 1], 1)
        v = lv.start_vector(mu)
        u = [lv.left_vector(l) for l in range(3)]
        e = np.zeros(m, dtype=np.complex128)
        e[0] = 1.0
        lkv = v.copy()
        for k in range(10):
            for l in range(3):
                lhs = w * c.n0 * np.vdot(c.z[l, :m], e)
                rhs = w * np.vdot(u[l], lkv)
                # scale: |w| ||u|| ||L^k v|| (the moments themselves can cancel)
                scale = w * np.linalg.norm(u[l]) * np.linalg.norm(lkv)
                assert abs(lhs - rhs) <= 1e-10 * scale
            e = t @ e
            lkv = lv.apply(lkv)


def test_p7_biorthogonality(c0_chains):
    for mu in range(3):
        nh = c0_chains["nh"][mu]
        g = np.array([[np.vdot(p, q) for q in nh.basis_q] for p in nh.basis_p])
        assert np.max(np.abs(g - np.eye(len(nh.basis_q)))) <= 1e-10
        pm = c0_chains["phm"][mu]
        g = np.array([[np.vdot(p, q) for q in pm.basis_q] for p in pm.basis_p])
        assert np.max(np.abs(g - np.eye(len(pm.basis_q)))) <= 1e-10
        ph = c0_chains["ph"][mu]
        k = 8
        nq = np.array([np.linalg.norm(q) for q in ph.basis_q[:k]])
        gj = np.array([[jdot(qi, qj) for qj in ph.basis_q[:k]] for qi in ph.basis_q[:k]])
        assert np.max(np.abs(gj - np.diag(ph.signs[:k])) / np.outer(nq, nq)) <= 1e-8
        # the PH recursion's alpha is real in exact arithmetic (J L is Hermitian on range(P_c))
        assert np.max(np.abs(ph.alpha.imag)) == 0.0


def test_first_step_from_an_eigenvector():
    """Started from an exact eigenvector a of the brute-force L (L a = lambda a), the NH
    recursion (Sec. 2.5) finds alpha_1 = lambda and a right residual r at rounding level;
    p_1 = q_1 is not a left eigenvector, so t = O(|lambda|) and beta_2 = sqrt|t^H r| is of
    order sqrt(eps) |lambda|.  A generic start vector has beta_2 of the order of the
    spectrum's width."""
    lv, ph = liouvillian("C0"), particle_hole("C0")
    ev, vec = np.linalg.eig(ph.L)
    i = int(np.argmax(np.abs(ev)))
    u = [lv.left_vector(l) for l in range(3)]
    co = lanczos_nh(lv.apply, lv.apply_adjoint, ph.to_br(vec[:, i]), u, 2)
    assert abs(co.alpha[0] - ev[i]) <= 1e-10 * abs(ev[i])
    assert co.beta[0] <= 1e-6 * abs(ev[i])
    gen = lanczos_nh(lv.apply, lv.apply_adjoint, lv.start_vector(0), u, 2)
    assert gen.beta[0] >= 1e-3 * abs(ev[i])


def test_p12_dense_vs_matrix_free():
    """NH and PHM agree step by step to rounding over 50 steps.  The J-metric PH
    is compared on the longitudinal chain (mu = z): for the transverse chains the
    start vector has nearly equal X and Y weight, ||q_1|| ~ 30 at unit J-norm, and
    r = L q - alpha q - gamma q' cancels catastrophically (alpha ~ +-200), so two
    correct codes part after a few steps; that conditioning is a property of the
    indefinite metric, not of either code.  Even on mu = z the left projections z
    amplify rounding-order differences ~1e5-fold over 20 steps (alpha, beta, gamma
    stay within ~3e-12), hence 1e-9 there."""
    lv, ph = liouvillian("C0"), particle_hole("C0")
    v = lv.start_vector(1)
    u = [lv.left_vector(l) for l in range(3)]
    va = ph.from_br(v)[0]
    ua = [ph.from_br(x)[0] for x in u]
    for flavor in ("nh", "ph", "phm"):
        if flavor == "nh":
            m, tol = 50, 1e-12
            a = lanczos_nh(lv.apply, lv.apply_adjoint, v, u, m)
            b = lanczos_nh(lambda x: ph.L @ x, lambda x: ph.L.conj().T @ x, va, ua, m)
        elif flavor == "phm":
            m, tol = 50, 1e-12
            a = lanczos_phm(lv.apply, v, u, m)
            b = lanczos_phm_dense(ph.L, ph.J, va, ua, m)
        else:
            m, tol = 20, 1e-9
            vz = lv.start_vector(2)
            a = lanczos_ph(lv.apply, vz, u, m)
            b = lanczos_ph_dense(ph.L, ph.J, ph.from_br(vz)[0], ua, m)
        for fa, fb in ((a.alpha, b.alpha), (a.beta, b.beta), (a.gamma, b.gamma), (a.z, b.z)):
            assert np.max(np.abs(fa - fb)) <= tol * np.max(np.abs(fb))


def lanczos_phm_dense(lmat, jvec, v, u, m):
    """Standard Hermitian Lanczos for L in the metric H = J L, written with explicit H."""
    hmat = jvec[:, None] * lmat
    n0 = np.sqrt(np.vdot(v, hmat @ v).real)
    q, qp, b = v / n0, np.zeros_like(v), 0.0
    from oracle.lanczos import Coefficients
    al, be = np.zeros(m, complex), np.zeros(m)
    z = np.zeros((3, m), complex)
    for j in range(m):
        a = lmat @ q
        al[j] = np.vdot(q, hmat @ a).real
        z[:, j] = [np.vdot(q, x) for x in u]
        r = a - al[j] * q - b * qp
        be[j] = np.sqrt(np.vdot(r, hmat @ r).real)
        qp, q, b = q, r / be[j], be[j]
    return Coefficients(al, be, be.astype(complex), z, n0, m, "ok")


def lanczos_ph_dense(lmat, jvec, v, u, m):
    """The same J-metric recursion written on the dense particle-hole basis."""
    c0 = np.vdot(v, jvec * v).real
    n0 = np.sqrt(abs(c0))
    s = np.sign(c0)
    q, qp, g = v / n0, np.zeros_like(v), 0.0
    from oracle.lanczos import Coefficients
    al, be, ga = np.zeros(m, complex), np.zeros(m), np.zeros(m, complex)
    z = np.zeros((3, m), complex)
    for j in range(m):
        a = lmat @ q
        al[j] = s * np.vdot(q, jvec * a).real
        z[:, j] = [np.vdot(q, x) for x in u]
        r = a - al[j] * q - g * qp
        c = np.vdot(r, jvec * r).real
        be[j] = np.sqrt(abs(c))
        sn = np.sign(c)
        ga[j] = s * sn * be[j]
        qp, q, s, g = q, r / be[j], sn, ga[j]
    return Coefficients(al, be, ga, z, n0, m, "ok")


@pytest.mark.parametrize("flavor", ["nh", "ph", "phm"])
def test_p3_chi0_closed_form(flavor):
    gs = ground_state("C0", 0)
    lv, ph = liouvillian("C0", 0), particle_hole("C0", 0)
    eta = 10.0 / HA_MEV
    w = gs.wk[0]
    mu = 0
    # closed form: w sum [<U|s_l|phi><phi|s_m|U>/(w+ieta-D^X) - (same on Y)/(w+ieta+D^Y)]
    va = ph.from_br(lv.start_vector(mu))[0]
    ua = [ph.from_br(lv.left_vector(l))[0] for l in range(3)]
    ref = np.zeros((3, len(OMEGAS)), dtype=np.complex128)
    for i, om in enumerate(OMEGAS):
        den = (om + 1j * eta) - ph.J * ph.D
        for l in range(3):
            ref[l, i] = w * np.sum(np.conj(ua[l]) * va / den)
    c = run_chain(lv, mu, 700, flavor)
    got = chi_thomas(c, OMEGAS, eta, w)
    tol = 1e-4 if flavor == "ph" else 1e-8
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref[mu])


def test_thomas_matches_banded(c0_chains):
    """Unpivoted Thomas vs pivoted banded LU.  They agree to rounding for the
    symmetric (PHM) and NH tridiagonals; the J-metric T alternates sign and is
    ill-conditioned without pivoting, so there only 1e-5 holds (the pivoted solve
    is the primary one, ``chi``)."""
    lv = liouvillian("C0")
    for flavor, tol in (("nh", 1e-12), ("phm", 1e-12), ("ph", 1e-5)):
        c = c0_chains[flavor][0]
        for eta in (10.0 / HA_MEV, 0.05):
            a = chi_thomas(c, OMEGAS, eta, lv.gs.wk[0], m=300)
            b = chi_banded(c, OMEGAS, eta, lv.gs.wk[0], m=300)
            assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))


def test_p8_collinear_symmetry():
    lv = liouvillian("C0", 3, True)
    eta = 0.05
    chi = np.array([chi_thomas(run_chain(lv, mu, 300, "nh"), OMEGAS, eta, lv.gs.wk[0])
                    for mu in range(3)])  # chi[mu][lam]
    scale = np.abs(chi).max()
    assert np.abs(chi[2][0]).max() <= 1e-12 * scale and np.abs(chi[0][2]).max() <= 1e-12 * scale
    assert np.abs(chi[2][1]).max() <= 1e-12 * scale and np.abs(chi[1][2]).max() <= 1e-12 * scale
    assert np.abs(chi[0][0] - chi[1][1]).max() <= 1e-8 * scale
    assert np.abs(chi[1][0] + chi[0][1]).max() <= 1e-8 * scale


def test_p9_sum_rule():
    """int_{-R}^{R} chi d omega -> -i pi w u^H v; the 1/omega tails leave a real
    remainder -2 w u^H L v / R (first moment), which is added back."""
    lv = liouvillian("C0")
    c = run_chain(lv, 0, 600, "nh")
    w = lv.gs.wk[0]
    eta = 0.05
    u = [lv.left_vector(l) for l in range(3)]
    v = lv.start_vector(0)
    exact = -1j * np.pi * w * np.array([np.vdot(x, v) for x in u])
    assert np.allclose(exact, -1j * np.pi * w * c.n0 * np.conj(c.z[:, 0]), rtol=1e-12)
    first = w * np.vdot(u[0], lv.apply(v))
    r = 400.0
    om = np.linspace(-r, r, 160001)
    integ = np.trapezoid(chi_thomas(c, om, eta, w), om, axis=1)
    assert abs(integ[0] + 2.0 * first / r - exact[0]) <= 1e-4 * abs(exact[0])


def _terminator_chi(coef, omegas, eta, w, itermax0, itermax, kind):
    """The extrapolated tail folded into the last computed diagonal entry by its
    backward continued fraction (what the GPU spectrum kernel evaluates)."""
    from oracle.spectrum import extrapolation_constants
    c = extrapolation_constants(coef, itermax0, kind)
    out = np.zeros((3, len(omegas)), dtype=np.complex128)
    for i, om in enumerate(omegas):
        zz = om + 1j * eta
        g = 0.0
        for j in range(itermax - 1, itermax0 - 1, -1):
            a, b, gm = c[j % 2]
            link = (b.real * gm) if j < itermax - 1 else 0.0
            g = 1.0 / (zz - a - link * g)
        m = itermax0
        d = zz - coef.alpha[:m].astype(complex)
        d[m - 1] -= coef.beta[m - 1] * coef.gamma[m - 1] * g
        ab = np.zeros((3, m), dtype=np.complex128)
        ab[0, 1:] = -coef.gamma[:m - 1]
        ab[1] = d
        ab[2, :-1] = -coef.beta[:m - 1]
        e1 = np.zeros(m, dtype=np.complex128)
        e1[0] = 1
        x = __import__("scipy.linalg").linalg.solve_banded((1, 1), ab, e1)
        out[:, i] = w * coef.n0 * (coef.z[:, :m].conj() @ x)
    return out


@pytest.mark.parametrize("kind", ["constant", "osc"])
def test_extrapolation_terminator_equals_extended_system(c0_chains, kind):
    """Folding the extrapolated tail into one diagonal entry (continued fraction)
    equals solving the explicitly extended system; 'no' equals truncation."""
    from oracle.spectrum import chi_extrapolated, extend_coefficients
    lv = liouvillian("C0")
    c = c0_chains["nh"][0]
    w = lv.gs.wk[0]
    eta = 10.0 / HA_MEV
    ref = chi_extrapolated(c, OMEGAS, eta, w, 60, 400, kind)
    got = _terminator_chi(c, OMEGAS, eta, w, 60, 400, kind)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    ext = extend_coefficients(c, 60, 400, kind)
    assert ext.steps == 400 and not ext.z[:, 60:].any()
    if kind == "constant":
        assert np.allclose(ext.beta[60:], ext.beta[60]) and np.allclose(ext.alpha[60:], ext.alpha[60])
    else:
        assert np.allclose(ext.beta[60::2], ext.beta[60]) and np.allclose(ext.beta[61::2], ext.beta[61])
    trunc = chi_extrapolated(c, OMEGAS, eta, w, 60, 400, "no")
    assert np.allclose(trunc, chi_banded(c, OMEGAS, eta, w, m=60), rtol=1e-12, atol=0)


def test_structure_factor_projector_pins():
    """S(q, w) = -Im Tr[P_perp chi]: for q along x it keeps chi_yy + chi_zz; it is
    invariant under a common rotation of q and chi (R chi R^T); the longitudinal
    part q^ chi q^ drops out (chi = q q^T c gives S = 0)."""
    from oracle.spectrum import structure_factor
    rng = np.random.default_rng(3)
    chi_lm = rng.normal(size=(3, 3, 7)) + 1j * rng.normal(size=(3, 3, 7))  # [lambda][mu][w]
    chi3 = np.transpose(chi_lm, (1, 0, 2))  # [mu][lambda][w]
    s = structure_factor(chi3, [2.0, 0.0, 0.0])
    assert np.allclose(s, -(chi_lm[1, 1] + chi_lm[2, 2]).imag, rtol=0, atol=1e-14)
    th = 0.7
    rot = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    rot = rot @ np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    q = np.array([0.3, -1.1, 0.4])
    chi_rot = np.einsum("ab,bcw,dc->adw", rot, chi_lm, rot)
    s1 = structure_factor(np.transpose(chi_lm, (1, 0, 2)), q)
    s2 = structure_factor(np.transpose(chi_rot, (1, 0, 2)), rot @ q)
    assert np.allclose(s1, s2, rtol=0, atol=1e-13)
    qh = q / np.linalg.norm(q)
    long_only = np.einsum("a,b,w->abw", qh, qh, chi_lm[0, 0])
    assert np.allclose(structure_factor(np.transpose(long_only, (1, 0, 2)), q), 0, atol=1e-14)

"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances:
* one Liouvillian application, FP64: relative L2 error <= 1e-12;
* one Liouvillian application, mixed (FP32 storage/arithmetic): <= 2e-5;
* Lanczos coefficients, FP64, NH and positive-definite PH: <= 1e-9 relative to
  the largest coefficient over 50 steps; J-metric PH over its first 12 steps on
  the longitudinal chain at 1e-7: its alternating tiny beta amplify the 1e-15
  differences of two correct FP64 codes by ~1e7 (the same spread appears between
  the oracle's matrix-free and dense runs);
* spectrum from identical coefficients: <= 1e-12 relative;
* chi(omega) end to end at eta = 10 meV, FP64: <= 1e-8 relative.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _cases import ground_state, liouvillian  # noqa: E402
from synth import random_br_vector  # noqa: E402


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_2203_01120_gb300 import Context, build
    build()
    c = Context(0)
    yield c
    c.close()


_slots = {}


def slot(ctx, name, mask=3, collinear=False):
    key = (name, mask, collinear)
    if key not in _slots:
        _slots[key] = ctx.load_ground_state(ground_state(name, mask, collinear))
    return _slots[key]


def apply_gpu(torch, ctx, q, x, adjoint=False, mixed=False):
    from paper_2203_01120_gb300 import TDLZ_FP64, TDLZ_MIXED
    dt = torch.complex64 if mixed else torch.complex128
    xt = torch.as_tensor(x, dtype=dt, device="cuda").contiguous()
    yt = torch.zeros_like(xt)
    ctx.apply_liouvillian(q, xt, yt, adjoint, TDLZ_MIXED if mixed else TDLZ_FP64)
    ctx.synchronize()
    return yt.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("name,mask", [("C0", 3), ("C0K", 0), ("C0K", 1), ("C0K", 2), ("C0K", 3),
                                       ("C0F", 3), ("C1", 3)])
def test_apply_fp64(torch, ctx, name, mask):
    q = slot(ctx, name, mask)
    lv = liouvillian(name, mask)
    x = random_br_vector(lv.gs, seed=7)
    y = apply_gpu(torch, ctx, q, x)
    ref = lv.apply(x)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= 1e-12, err
    # padding stays zero
    for k in range(lv.gs.nk):
        assert not y[:, k, :, :, lv.gs.npw_kq[k]:].any()


def test_apply_adjoint_fp64(torch, ctx):
    q = slot(ctx, "C0K")
    lv = liouvillian("C0K")
    x = random_br_vector(lv.gs, seed=8)
    y = apply_gpu(torch, ctx, q, x, adjoint=True)
    ref = lv.apply_adjoint(x)
    assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("name", ["C0K", "C0F", "C1"])
def test_apply_mixed(torch, ctx, name):
    q = slot(ctx, name)
    lv = liouvillian(name)
    x = random_br_vector(lv.gs, seed=9)
    y = apply_gpu(torch, ctx, q, x, mixed=True)
    ref = lv.apply(x)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= 2e-5, err


@pytest.mark.parametrize("env", [{"TDLZ_TC": "0"}])
@pytest.mark.parametrize("name", ["C0K", "C1"])
def test_apply_mixed_alternative_paths(torch, ctx, name, env, monkeypatch):
    """The mixed-precision Liouvillian through its alternative code path (chosen per
    q-slot at load): the CUDA-core reduction GEMMs in place of the tensor-core ones
    (the fused plane stages have their own file, test_gpu_planes.py)."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    q = ctx.load_ground_state(ground_state(name))
    lv = liouvillian(name)
    x = random_br_vector(lv.gs, seed=9)
    y = apply_gpu(torch, ctx, q, x, mixed=True)
    ref = lv.apply(x)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err <= 2e-5, err


def test_apply_is_deterministic(torch, ctx):
    q = slot(ctx, "C1")
    lv = liouvillian("C1")
    x = random_br_vector(lv.gs, seed=10)
    a = apply_gpu(torch, ctx, q, x)
    b = apply_gpu(torch, ctx, q, x)
    assert np.array_equal(a, b)


def _oracle_chain(name, mu, steps, flavor, mask=3):
    from oracle.lanczos import run_chain
    return run_chain(liouvillian(name, mask), mu, steps, flavor)


@pytest.mark.parametrize("flavor,mu,steps,tol", [("nh", 0, 50, 1e-9), ("phm", 0, 50, 1e-9),
                                                 ("nh", 2, 50, 1e-9), ("ph", 2, 12, 1e-7)])
def test_lanczos_fp64(torch, ctx, flavor, mu, steps, tol):
    q = slot(ctx, "C1")
    got = ctx.lanczos_run([q], [mu], steps, flavor)
    ref = _oracle_chain("C1", mu, steps, flavor)
    assert got["status"][0] == 0 and got["steps_done"][0] == steps
    assert abs(got["n0"][0] - ref.n0) <= 1e-12 * ref.n0
    for key, r in (("alpha", ref.alpha), ("beta", ref.beta), ("gamma", ref.gamma)):
        g = got[key][0]
        assert np.max(np.abs(g - r)) <= tol * np.max(np.abs(r)), key
    assert np.max(np.abs(got["z"][0] - ref.z)) <= tol * np.max(np.abs(ref.z))


def test_spectrum_matches_oracle_on_same_coefficients(torch, ctx):
    from oracle.lanczos import Coefficients
    from oracle.spectrum import chi_banded, omega_grid_mev, HA_MEV
    q = slot(ctx, "C1")
    got = ctx.lanczos_run([q, q], [0, 2], 50, "nh")
    chi = ctx.spectrum(got, 0.0, 400.0, 0.5, 10.0, units=1)
    om = omega_grid_mev(0.0, 400.0, 0.5) / HA_MEV
    for c in range(2):
        co = Coefficients(got["alpha"][c], got["beta"][c], got["gamma"][c], got["z"][c],
                          got["n0"][c], int(got["steps_done"][c]), "ok")
        ref = chi_banded(co, om, 10.0 / HA_MEV, got["wk"][c])
        assert chi.shape == (2, 3, len(om))
        assert np.max(np.abs(chi[c] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("flavor", ["nh", "phm"])
def test_chi_end_to_end_fp64(torch, ctx, flavor):
    """Target tolerance: chi at eta = 10 meV within 1e-8 of the oracle (C1, 50 steps)."""
    from oracle.spectrum import chi_banded, omega_grid_mev, HA_MEV
    q = slot(ctx, "C1")
    got = ctx.lanczos_run([q], [1], 50, flavor)
    chi = ctx.spectrum(got, 0.0, 2000.0, 2.0, 10.0, units=1)[0]
    ref_c = _oracle_chain("C1", 1, 50, flavor)
    om = omega_grid_mev(0.0, 2000.0, 2.0) / HA_MEV
    ref = chi_banded(ref_c, om, 10.0 / HA_MEV, liouvillian("C1").gs.wk[0])
    err = np.linalg.norm(chi - ref) / np.linalg.norm(ref[1])
    assert err <= 1e-8, err


def test_invalid_inputs_rejected(torch, ctx):
    import dataclasses
    from paper_2203_01120_gb300 import TdlzError
    gs = ground_state("C0")
    bad_q = dataclasses.replace(gs, q=np.zeros(3))
    with pytest.raises(TdlzError) as e:
        ctx.load_ground_state(bad_q)
    assert e.value.status == 1
    bad_npw = dataclasses.replace(gs, npw_kq=gs.npw_kq + gs.npwx)
    with pytest.raises(TdlzError):
        ctx.load_ground_state(bad_npw)
    d = gs.dnl.copy()
    d[0, 1] += 0.1
    with pytest.raises(TdlzError):
        ctx.load_ground_state(dataclasses.replace(gs, dnl=d))
    q = slot(ctx, "C0")
    x = __import__("torch").zeros(10, dtype=__import__("torch").complex128, device="cuda")
    with pytest.raises(TdlzError):
        ctx.apply_liouvillian(q, x, x)  # overlapping x, y


@pytest.mark.parametrize("flavor", ["nh", "phm"])
def test_grouped_chains_equal_single_chains(torch, ctx, flavor):
    """Chains of one q-slot advance in one stacked Liouvillian pass; each must match
    the same chain run alone (C1, FP64, 20 steps)."""
    q = slot(ctx, "C1")
    grouped = ctx.lanczos_run([q, q, q], [0, 1, 2], 20, flavor)
    for c in range(3):
        alone = ctx.lanczos_run([q], [c], 20, flavor)
        for key in ("alpha", "beta", "gamma", "z"):
            a, b = grouped[key][c], alone[key][0]
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), (c, key)


@pytest.mark.parametrize("kind", ["constant", "osc"])
def test_spectrum_extrapolation_matches_oracle(torch, ctx, kind):
    """Extrapolated chi (itermax0 = 30 computed, itermax = 2000) against the oracle's
    explicitly extended system."""
    from oracle.lanczos import Coefficients
    from oracle.spectrum import chi_extrapolated, omega_grid_mev, HA_MEV
    q = slot(ctx, "C1")
    got = ctx.lanczos_run([q], [0], 40, "nh")
    chi = ctx.spectrum(got, 0.0, 1000.0, 2.0, 10.0, units=1, itermax0=30, itermax=2000,
                       extrapolation=kind)[0]
    co = Coefficients(got["alpha"][0], got["beta"][0], got["gamma"][0], got["z"][0],
                      got["n0"][0], int(got["steps_done"][0]), "ok")
    om = omega_grid_mev(0.0, 1000.0, 2.0) / HA_MEV
    ref = chi_extrapolated(co, om, 10.0 / HA_MEV, got["wk"][0], 30, 2000, kind)
    assert np.max(np.abs(chi - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("flavor,prec", [("nh", 0), ("phm", 0), ("nh", 1), ("ph", 1)])
def test_restart_resumes_bitwise(torch, ctx, flavor, prec):
    """Save after 12 steps, restore into a fresh chain set of larger capacity,
    continue to 30: identical coefficients to an uninterrupted 30-step run."""
    q = slot(ctx, "C1")
    straight = ctx.lanczos_run([q, q], [0, 2], 30, flavor, prec)
    a = ctx.chain_create([q, q], [0, 2], 12, flavor, prec)
    a.advance(12)
    image = a.save()
    a.close()
    b = ctx.chain_create([q, q], [0, 2], 30, flavor, prec)
    b.restore(image)
    b.advance(18)
    resumed = b.read()
    b.close()
    for key in ("alpha", "beta", "gamma", "z", "n0", "steps_done", "status"):
        assert np.array_equal(resumed[key], straight[key]), key


@pytest.mark.parametrize("flavor,prec", [("nh", 1), ("ph", 0), ("phm", 0), ("phm", 1)])
def test_graph_replay_matches_eager_steps(torch, ctx, flavor, prec):
    """Steps replayed from the captured two-step CUDA graph (advance(n >= 4)) give the
    same coefficients, bit for bit, as one eager launch sequence per step; an odd
    split (5 + 8) forces a re-capture with the other vector rotation."""
    q = slot(ctx, "C1")
    eager = ctx.chain_create([q, q], [0, 1], 13, flavor, prec)
    for _ in range(13):
        eager.advance(1)
    ref = eager.read()
    eager.close()
    for split in ((13,), (5, 8)):
        g = ctx.chain_create([q, q], [0, 1], 13, flavor, prec)
        for n in split:
            g.advance(n)
        got = g.read()
        g.close()
        for key in ("alpha", "beta", "gamma", "z", "n0", "steps_done", "status"):
            assert np.array_equal(got[key], ref[key]), (split, key)


def test_structure_factor_matches_oracle(torch, ctx):
    """S(q, w) = -Im Tr[P_perp chi] from the three chains mu = x, y, z of one q-slot."""
    from oracle.spectrum import structure_factor
    q = slot(ctx, "C1")
    got = ctx.lanczos_run([q, q, q], [0, 1, 2], 30, "nh")
    chi = ctx.spectrum(got, 0.0, 1000.0, 5.0, 10.0, units=1)  # [mu][lambda][w]
    qv = ground_state("C1").q
    s = ctx.structure_factor(chi, qv)
    ref = structure_factor(chi, qv)
    assert np.max(np.abs(s - ref)) <= 1e-13 * np.max(np.abs(ref))
    from paper_2203_01120_gb300 import TdlzError
    with pytest.raises(TdlzError):
        ctx.structure_factor(chi, [0.0, 0.0, 0.0])


def test_multi_q_chain_set_equals_separate_runs(torch, ctx):
    """Batched form: chains on two q-slots (q and 2q) advance in one chain set (one
    group per slot, both replayed from one captured graph) and reproduce the
    single-slot runs coefficient for coefficient."""
    from synth import make_ground_state
    q1 = slot(ctx, "C0K")
    q2 = ctx.load_ground_state(make_ground_state("C0K", q_2pi_a=(0.2, 0.0, 0.0)))
    both = ctx.lanczos_run([q1, q2, q1, q2], [0, 0, 2, 2], 16, "nh")
    for c, (qs, mu) in enumerate([(q1, 0), (q2, 0), (q1, 2), (q2, 2)]):
        alone = ctx.lanczos_run([qs], [mu], 16, "nh")
        for key in ("alpha", "beta", "gamma", "z", "n0"):
            a, b = both[key][c], alone[key][0]
            assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b)), (c, key)


def test_larmor_mode_on_gpu(torch, ctx):
    """The self-consistent collinear model with a uniform external field b_ext = 0.05
    (no spin-orbit coupling): the GPU Liouvillian maps the brute-force Larmor
    eigenvector to 2 b_ext times itself, and the NH chain started from sigma_x U has
    a Ritz value at 2 b_ext."""
    from synth import make_ground_state
    from oracle.liouvillian import Liouvillian
    from _bruteforce import ParticleHole
    gs = make_ground_state("C0", collinear=True, kernel_mask=2, q_2pi_a=(1e-4, 0.0, 0.0),
                           self_consistent=True, b_ext=0.05)
    q = ctx.load_ground_state(gs)
    lv = Liouvillian(gs)
    ph = ParticleHole(gs, lv.fxc)
    ev, vec = np.linalg.eig(ph.L)
    i = int(np.argmin(np.abs(ev - 0.1)))
    x = ph.to_br(vec[:, i])
    y = apply_gpu(torch, ctx, q, x)
    assert np.linalg.norm(y - 0.1 * x) <= 1e-7 * np.linalg.norm(x)
    got = ctx.lanczos_run([q], [0], 30, "nh")
    m = int(got["steps_done"][0])
    t = np.diag(got["alpha"][0][:m]) + np.diag(got["beta"][0][:m - 1], -1) + np.diag(
        got["gamma"][0][:m - 1], 1)
    ritz = np.linalg.eigvals(t)
    assert np.min(np.abs(ritz - 0.1)) <= 1e-6, np.sort(np.abs(ritz - 0.1))[:3]


@pytest.mark.parametrize("name", ["C0K", "C1"])
def test_autotuned_shapes_change_no_result(torch, name, monkeypatch):
    """The autotuner only picks among launch shapes that compute identical results:
    a context with TDLZ_AUTOTUNE=0 (default shapes) and a tuning one give bitwise
    equal L x (FP64 and mixed) and Lanczos coefficients; the tuning context reports
    its decisions."""
    from paper_2203_01120_gb300 import Context, TDLZ_MIXED
    lv = liouvillian(name)
    x = random_br_vector(lv.gs, seed=31)
    out = []
    for env in ("0", "1"):
        monkeypatch.setenv("TDLZ_AUTOTUNE", env)
        c = Context(0)
        try:
            q = c.load_ground_state(ground_state(name))
            ys = [apply_gpu(torch, c, q, x), apply_gpu(torch, c, q, x, mixed=True)]
            chains = c.lanczos_run([q, q], [0, 2], 12, "nh", TDLZ_MIXED)
            report = c.autotune_report()
        finally:
            c.close()
        out.append((ys, chains, report))
    (y0, c0, r0), (y1, c1, r1) = out
    assert r0 == {} and len(r1) >= 1, r1
    for a, b in zip(y0, y1):
        assert np.array_equal(a, b)
    for key in ("alpha", "beta", "gamma", "z"):
        assert np.array_equal(c0[key], c1[key]), key


def test_restart_rejects_mismatched_image(torch, ctx):
    from paper_2203_01120_gb300 import TdlzError
    q = slot(ctx, "C1")
    a = ctx.chain_create([q], [0], 5, "nh")
    a.advance(2)
    image = a.save()
    a.close()
    b = ctx.chain_create([q], [1], 5, "nh")  # different mu
    with pytest.raises(TdlzError):
        b.restore(image)
    b.close()
    c = ctx.chain_create([q], [0], 3, "nh")  # smaller capacity
    with pytest.raises(TdlzError):
        c.restore(image)
    c.close()


def test_tensor_core_reductions_above_64_bands(torch, monkeypatch):
    """P_c's reduction <U_kq|h> with more than 64 occupied bands (2M > 128 rows, the
    CrI3-shaped workloads' 70) runs the transposed tensor-core form (the MMA's M = 128
    stacked rows of h, its N = the 2M rows of [Re; Im] of U_kq): the C1 grid with 72
    random orthonormal occupied states, mixed L x against the oracle (<= 2e-5) and against
    the CUDA-core contractions (TDLZ_TC=0, <= 1e-5)."""
    from paper_2203_01120_gb300 import Context, TDLZ_MIXED
    from synth import make_ground_state
    from oracle.liouvillian import Liouvillian
    gs = make_ground_state("C1", solver="random", nocc=72)
    x = random_br_vector(gs, seed=71)
    ref = Liouvillian(gs).apply(x)
    ys = []
    for tc in ("1", "0"):
        monkeypatch.setenv("TDLZ_TC", tc)
        c = Context(0)
        try:
            q = c.load_ground_state(gs)
            xt = torch.as_tensor(x, dtype=torch.complex64, device="cuda").contiguous()
            yt = torch.zeros_like(xt)
            c.apply_liouvillian(q, xt, yt, False, TDLZ_MIXED)
            c.synchronize()
            ys.append(yt.cpu().numpy().astype(np.complex128))
        finally:
            c.close()
    y_tc, y_cc = ys
    assert np.linalg.norm(y_tc - ref) <= 2e-5 * np.linalg.norm(ref)
    assert np.linalg.norm(y_tc - y_cc) <= 1e-5 * np.linalg.norm(ref)


def _c3_grid_small():
    from synth import make_ground_state
    return make_ground_state("C3", solver="random", kgrid=(2, 1, 1), nocc=6)


@pytest.mark.parametrize("ctas,in_tma", [("3", "0"), ("2", "0"), ("1", "0"), ("2", "1")])
@pytest.mark.parametrize("case", ["C0K", "C1", "C1-72", "C3grid"])
def test_update_gemm_images_equal_register_staging(torch, monkeypatch, case, ctas, in_tma):
    """The tensor-core updates of V_NL and P_c read precomputed TF32 operand images with
    bulk and tensor copies (the default; TDLZ_TC_IMG=0 keeps the register-staged kernel).
    Same operand values, same MMA order, same epilogue: mixed L x, its adjoint and 6 NH
    Lanczos steps (replayed from a captured graph) are bit for bit those of the
    register-staged kernel.  The cases cover the In tile read in the epilogue after an L2
    prefetch (the default) and fetched with one tensor copy per CTA (TDLZ_NN_IN_TMA=1:
    P_c's rows always, V_NL's on the 45x45x144 grid, whose spheres have an even number of
    plane waves per component), 72 bands (row blocks) and the shared-memory sizings for
    one, two or three CTAs per SM (TDLZ_NN_CTAS; fewer CTAs keep more K tiles in
    flight)."""
    from paper_2203_01120_gb300 import Context, TDLZ_MIXED
    from synth import make_ground_state
    if case == "C3grid":
        gs = _c3_grid_small()
    elif case == "C1-72":
        gs = make_ground_state("C1", solver="random", nocc=72)
    else:
        gs = ground_state(case)
    x = random_br_vector(gs, seed=81)
    monkeypatch.setenv("TDLZ_NN_CTAS", ctas)
    monkeypatch.setenv("TDLZ_NN_IN_TMA", in_tma)
    out = []
    for img in ("0", "1"):
        monkeypatch.setenv("TDLZ_TC_IMG", img)
        c = Context(0)
        try:
            q = c.load_ground_state(gs)
            ys = []
            for adjoint in (False, True):
                xt = torch.as_tensor(x, dtype=torch.complex64, device="cuda").contiguous()
                yt = torch.zeros_like(xt)
                c.apply_liouvillian(q, xt, yt, adjoint, TDLZ_MIXED)
                c.synchronize()
                ys.append(yt.cpu().numpy())
            chains = c.lanczos_run([q, q], [0, 2], 6, "nh", TDLZ_MIXED)
        finally:
            c.close()
        out.append((ys, chains))
    (y0, c0), (y1, c1) = out
    for a, b in zip(y0, y1):
        assert np.array_equal(a, b)
    for key in ("alpha", "beta", "gamma", "z"):
        assert np.array_equal(c0[key], c1[key]), key


def test_update_gemm_images_abort_path(torch, monkeypatch):
    """Every bounded wait of the tensor-core GEMMs (including the image-fed update's
    copy, MMA-commit and In waits) reports expiry once it has completed
    (TDLZ_TEST_INJECT_TC_TIMEOUT large): each CTA drains its copies and MMAs, releases
    TMEM and the call returns TDLZ_ERR_TIMEOUT; a new context (injection cleared) then
    computes L x within the mixed tolerance of the oracle."""
    from paper_2203_01120_gb300 import Context, TdlzError, TDLZ_MIXED
    lv = liouvillian("C1")
    x = random_br_vector(lv.gs, seed=83)

    def apply(c, q):
        xt = torch.as_tensor(x, dtype=torch.complex64, device="cuda").contiguous()
        yt = torch.zeros_like(xt)
        c.apply_liouvillian(q, xt, yt, False, TDLZ_MIXED)
        c.synchronize()
        return yt.cpu().numpy().astype(np.complex128)

    monkeypatch.setenv("TDLZ_TC", "1")
    monkeypatch.setenv("TDLZ_TEST_INJECT_TC_TIMEOUT", str(1 << 30))
    c = Context(0)
    try:
        q = c.load_ground_state(lv.gs)
        with pytest.raises(TdlzError) as e:
            apply(c, q)
        assert e.value.status == 7  # TDLZ_ERR_TIMEOUT
    finally:
        c.close()
    monkeypatch.setenv("TDLZ_TEST_INJECT_TC_TIMEOUT", "0")
    c = Context(0)
    try:
        q = c.load_ground_state(lv.gs)
        ref = lv.apply(x)
        assert np.linalg.norm(apply(c, q) - ref) <= 2e-5 * np.linalg.norm(ref)
    finally:
        c.close()


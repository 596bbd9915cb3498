"""The 4x4 generalised susceptibility through the GPU path: chains started from the
charge perturbation (mu = 3) and the charge left vector recorded as the fourth z
(ncomp = 4), against the oracle (whose charge vectors are pinned in
tests/test_oracle_charge.py).

* FP64 coefficients (alpha, beta, gamma, all four z) of NH and PHM chains for every
  column mu = x, y, z, charge on C1, 50 steps: <= 1e-9 of the oracle's;
* the 4x4 chi(omega) at eta = 10 meV from the GPU spectrum: <= 1e-8 of the oracle's;
* mixed precision (NH, 50 steps): chi within 1e-4 of the oracle's per column (after
  checking that the oracle is stable there under FP32-size perturbations);
* a chain set mixing spin and charge columns restarts bit for bit, an image is refused
  by a chain set of the other ncomp, and the allocation-free spectrum equals
  tdlz_spectrum for ncomp = 4.
"""

import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _cases import ground_state, liouvillian  # noqa: E402

ETA_MEV = 10.0


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


@functools.lru_cache(maxsize=None)
def slot_c1(ctx):
    return ctx.load_ground_state(ground_state("C1"))


@functools.lru_cache(maxsize=None)
def oracle_chain(mu, steps, flavor):
    from oracle.lanczos import run_chain
    return run_chain(liouvillian("C1"), mu, steps, flavor, ncomp=4)


@pytest.mark.parametrize("flavor", ["nh", "phm"])
def test_fp64_coefficients_all_columns(torch, ctx, flavor):
    q = slot_c1(ctx)
    got = ctx.lanczos_run([q] * 4, [0, 1, 2, 3], 50, flavor, ncomp=4)
    assert got["z"].shape[1] == 4
    for mu in range(4):
        ref = oracle_chain(mu, 50, flavor)
        assert got["status"][mu] == 0 and got["steps_done"][mu] == 50, mu
        assert abs(got["n0"][mu] - ref.n0) <= 1e-12 * ref.n0
        for key, r in (("alpha", ref.alpha), ("beta", ref.beta), ("gamma", ref.gamma)):
            assert np.max(np.abs(got[key][mu] - r)) <= 1e-9 * np.max(np.abs(r)), (mu, key)
        assert np.max(np.abs(got["z"][mu] - ref.z)) <= 1e-9 * np.max(np.abs(ref.z)), mu


def test_fp64_chi_4x4(torch, ctx):
    from oracle.spectrum import HA_MEV, chi_banded, omega_grid_mev
    q = slot_c1(ctx)
    got = ctx.lanczos_run([q] * 4, [0, 1, 2, 3], 50, "nh", ncomp=4)
    chi = ctx.spectrum(got, 0.0, 2000.0, 2.0, ETA_MEV, units=1)  # [mu][lambda][omega]
    assert chi.shape[:2] == (4, 4)
    om = omega_grid_mev(0.0, 2000.0, 2.0) / HA_MEV
    w = liouvillian("C1").gs.wk[0]
    for mu in range(4):
        ref = chi_banded(oracle_chain(mu, 50, "nh"), om, ETA_MEV / HA_MEV, w)
        assert np.linalg.norm(chi[mu] - ref) <= 1e-8 * np.linalg.norm(ref[mu]), mu


def test_mixed_chi_4x4_against_oracle(torch, ctx):
    from paper_2203_01120_gb300 import TDLZ_MIXED
    from oracle.lanczos import lanczos_nh
    from oracle.spectrum import HA_MEV, chi_banded, omega_grid_mev
    lv = liouvillian("C1")
    om = omega_grid_mev(0.0, 100.0, 0.1) / HA_MEV
    u = [lv.left_vector(l) for l in range(4)]
    q = slot_c1(ctx)
    got = ctx.lanczos_run([q] * 4, [0, 1, 2, 3], 50, "nh", TDLZ_MIXED, ncomp=4)
    assert not np.any(got["status"])
    chi = ctx.spectrum(got, 0.0, 100.0, 0.1, ETA_MEV, units=1)
    for mu in range(4):
        ref = chi_banded(oracle_chain(mu, 50, "nh"), om, ETA_MEV / HA_MEV, lv.gs.wk[0])
        # conditioning: the oracle's own chi under a 1e-7 relative start perturbation
        v = lv.start_vector(mu)
        rng = np.random.default_rng(200 + mu)
        d = rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)
        vp = v + 1e-7 * np.linalg.norm(v) * d / np.linalg.norm(d)
        refp = chi_banded(lanczos_nh(lv.apply, lv.apply_adjoint, vp, u, 50), om,
                          ETA_MEV / HA_MEV, lv.gs.wk[0])
        norm = np.linalg.norm(ref[mu])
        spread = np.linalg.norm(refp - ref, axis=1).max() / norm
        assert spread <= 2e-5, (mu, spread)
        err = np.linalg.norm(chi[mu] - ref, axis=1).max() / norm
        assert err <= 1e-4, (mu, err, spread)


def test_restart_and_noalloc_with_charge(torch, ctx):
    from paper_2203_01120_gb300 import TdlzError
    q = slot_c1(ctx)
    straight = ctx.lanczos_run([q, q], [3, 0], 20, "nh", ncomp=4)
    a = ctx.chain_create([q, q], [3, 0], 8, "nh", ncomp=4)
    a.advance(8)
    image = a.save()
    a.close()
    b = ctx.chain_create([q, q], [3, 0], 20, "nh", ncomp=4)
    b.restore(image)
    b.advance(12)
    resumed = b.read()
    b.close()
    for key in ("alpha", "beta", "gamma", "z", "n0", "steps_done", "status"):
        assert np.array_equal(resumed[key], straight[key]), key
    c = ctx.chain_create([q, q], [3, 0], 20, "nh", ncomp=3)
    with pytest.raises(TdlzError) as e:
        c.restore(image)
    assert e.value.status == 1
    c.close()
    # the allocation-free spectrum on device copies of the coefficients
    ref = ctx.spectrum(straight, 0.0, 500.0, 1.0, ETA_MEV, units=1)
    dev = {k: torch.as_tensor(np.ascontiguousarray(straight[k]), device="cuda")
           for k in ("alpha", "beta", "gamma", "z", "n0", "wk")}
    dev["steps_done"] = torch.as_tensor(straight["steps_done"], dtype=torch.int32, device="cuda")
    out = torch.zeros(ref.shape, dtype=torch.complex128, device="cuda")
    ctx.spectrum_noalloc(dev, 0.0, 500.0, 1.0, ETA_MEV, 1, out)
    ctx.synchronize()
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))

"""Mixed precision against the FP64 oracle at the level of chi(omega).

The mixed path (FP32 vectors and arithmetic, 3xTF32 tensor-core contractions, FP64
Lanczos scalars and spectrum) is required to give chi(omega) within 1e-4 of the FP64
oracle.  Error of a column mu: e_lambda_mu = ||chi_mixed - chi_oracle||_2 over the
omega grid, divided by ||chi_oracle[mu][mu]||_2 (off-diagonal components can be many
orders smaller than the diagonal one); the test takes the largest over lambda.

The comparison is only meaningful where the FP64 continued fraction itself is stable
under perturbations of FP32 size.  On C1 at eta = 10 meV a relative perturbation of
1e-7 of the start vector changes the oracle's own NH chi by ~1e-7 (0-100 meV) after
100 steps, but by 0.5% and 110% (0-3 eV, across the lowest poles near 0.89 eV) after
200 steps, once finite-precision Lanczos has lost biorthogonality: no FP32
computation can be held to 1e-4 there.  So each case first checks that the oracle's
chi moves by at most a fifth of the case's bound under that perturbation (the case
can resolve errors at the bound), then bounds the mixed chi:
* on the benchmark's grid, 0-100 meV in 0.1 meV steps (the chi error of the
  configuration), within 1e-4: NH over 100 steps (twice C1's configured 50), PHM over
  50 (over 100 steps its mixed error was measured at 1.6e-4 against an oracle spread
  of 7e-7: the bound is missed there);
* across the lowest poles, 0-3000 meV in 1 meV steps over 50 steps, within 1e-3: near
  a pole chi changes by (dE / eta) of itself for a shift dE of the pole, and the FP32
  application error (~1e-6 of ||L|| ~ 10 eV per step) shifts poles by ~1e-5 eV, i.e.
  ~1e-3 eta (measured: 5.9e-4 for the NH z column, whose oracle spread there is 5e-5).
"""

import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _cases import ground_state, liouvillian  # noqa: E402

ETA_MEV = 10.0
GRID_BENCH, GRID_POLES = (0.0, 100.0, 0.1), (0.0, 3000.0, 1.0)
CASES = [("nh", 100, GRID_BENCH, 1e-4), ("phm", 50, GRID_BENCH, 1e-4),
         ("nh", 50, GRID_POLES, 1e-3), ("phm", 50, GRID_POLES, 1e-3)]


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


def _chain(lv, v, steps, flavor):
    from oracle.lanczos import lanczos_nh, lanczos_phm
    u = [lv.left_vector(l) for l in range(3)]
    if flavor == "nh":
        return lanczos_nh(lv.apply, lv.apply_adjoint, v, u, steps)
    return lanczos_phm(lv.apply, v, u, steps)


@functools.lru_cache(maxsize=None)
def oracle_chi(flavor, steps, grid, perturb):
    """chi[mu][lambda][omega] of the oracle; perturb > 0 adds a seeded relative
    perturbation of that size to each start vector."""
    from oracle.spectrum import HA_MEV, chi_banded, omega_grid_mev
    lv = liouvillian("C1")
    om = omega_grid_mev(*grid) / HA_MEV
    out = []
    for mu in range(3):
        v = lv.start_vector(mu)
        if perturb:
            rng = np.random.default_rng(100 + mu)
            d = rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)
            v = v + perturb * np.linalg.norm(v) * d / np.linalg.norm(d)
        c = _chain(lv, v, steps, flavor)
        out.append(chi_banded(c, om, ETA_MEV / HA_MEV, lv.gs.wk[0]))
    return np.stack(out)


def column_errors(chi, ref):
    return [float(np.linalg.norm(chi[mu] - ref[mu], axis=1).max() / np.linalg.norm(ref[mu][mu]))
            for mu in range(3)]


@pytest.mark.parametrize("flavor,steps,grid,tol", CASES)
def test_mixed_chi_against_oracle(torch, ctx, flavor, steps, grid, tol):
    from paper_2203_01120_gb300 import TDLZ_MIXED
    ref = oracle_chi(flavor, steps, grid, 0.0)
    spread = max(column_errors(oracle_chi(flavor, steps, grid, 1e-7), ref))
    assert spread <= tol / 5, ("oracle chi not stable at FP32-size perturbations", spread)
    q = ctx.load_ground_state(ground_state("C1"))
    got = ctx.lanczos_run([q, q, q], [0, 1, 2], steps, flavor, TDLZ_MIXED)
    assert not np.any(got["status"]) and np.all(got["steps_done"] == steps)
    chi = ctx.spectrum(got, *grid, ETA_MEV, units=1)  # [mu][lambda][omega]
    errs = column_errors(chi, ref)
    assert max(errs) <= tol, (errs, spread)

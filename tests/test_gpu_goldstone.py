"""Goldstone check through the GPU path (the model and the brute-force reference are
those of tests/test_oracle_goldstone.py: two electrons per cell, spontaneously
polarised by the self-consistent Slater exchange, q = 0.01 2pi/a).

* The FP64 GPU Liouvillian maps the brute-force eigenvector of the lowest mode to
  omega times itself, without spin-orbit coupling (omega = 2.4e-6 Ha, on its way to
  zero as q^2) and with it (omega = 5.3e-4 Ha, the gap).
* The FP64 NH chain started from sigma_x U has Ritz values at both members of the pair
  +-omega after 200 steps (the start vector lies almost wholly in that pair, and the
  chain resolves the pair once its small remainder elsewhere has been deflated).
"""

import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

Q = 0.01


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
def case(soc: bool):
    from synth import make_ground_state
    from oracle.liouvillian import Liouvillian
    from _bruteforce import ParticleHole
    gs = make_ground_state("CG", collinear=not soc, self_consistent=True, b_ext=0.0,
                           q_2pi_a=(Q, 0.0, 0.0))
    ph = ParticleHole(gs, Liouvillian(gs).fxc)
    ev, vec = np.linalg.eig(ph.L)
    order = np.argsort(np.abs(ev))[:2]
    order = order[np.argsort(ev[order].real)]
    return gs, ph, ev[order].real, vec[:, order]


@pytest.mark.parametrize("soc", [False, True])
def test_lowest_mode_eigenpair_on_gpu(torch, ctx, soc):
    from paper_2203_01120_gb300 import TDLZ_FP64
    gs, ph, pair, vec = case(soc)
    q = ctx.load_ground_state(gs)
    for i in range(2):
        x = ph.to_br(vec[:, i])
        xt = torch.as_tensor(x, dtype=torch.complex128, device="cuda").contiguous()
        yt = torch.zeros_like(xt)
        ctx.apply_liouvillian(q, xt, yt, False, TDLZ_FP64)
        ctx.synchronize()
        y = yt.cpu().numpy()
        assert np.linalg.norm(y - pair[i] * x) <= 1e-10 * np.linalg.norm(x), (soc, i)


@pytest.mark.parametrize("soc", [False, True])
def test_nh_chain_ritz_values_at_the_pair(torch, ctx, soc):
    from paper_2203_01120_gb300 import TDLZ_FP64
    gs, _, pair, _ = case(soc)
    q = ctx.load_ground_state(gs)
    got = ctx.lanczos_run([q], [0], 200, "nh", TDLZ_FP64)
    m = int(got["steps_done"][0])
    assert got["status"][0] == 0 and m == 200
    t = (np.diag(got["alpha"][0][:m]) + np.diag(got["beta"][0][:m - 1], -1)
         + np.diag(got["gamma"][0][:m - 1], 1))
    ritz = np.linalg.eigvals(t)
    for w in pair:
        assert np.min(np.abs(ritz - w)) <= 1e-9, (soc, w, np.sort(np.abs(ritz - w))[:2])

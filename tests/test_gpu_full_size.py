"""GPU parity at the full C2 workload size (FFT 36x36x96, ~5000 plane waves per
spinor component, 4x4 k points, 40 occupied bands, 8 atoms x 8 KB projectors).

The oracle cannot apply L to a whole C2 vector in seconds, so the checks are:
* sampled outputs: the oracle's L x at three k points (the response density it
  needs still sums over all sixteen), element by element against the FP64 and
  the mixed GPU outputs at those k points;
* properties that hold at any size: the mixed output against the FP64 output
  everywhere, zero padding, and the pseudo-Hermiticity of L on the range of the
  empty-manifold projectors (a^H J L b = conj(b^H J L a)) over whole vectors;
* the launch configuration that is timed on C2 (three NH chains mu = x, y, z of
  one q-slot advancing together, mixed precision, graph replay) against each
  chain run alone.

The occupied states are random orthonormal spinors on the C2 spheres (the
operator L is defined for any orthonormal occupied set and any band energies;
the eigensolver is skipped to keep the test short).  Tolerances as in the small
cases: FP64 <= 1e-12, mixed <= 2e-5 (relative L2 over the compared elements).
"""

import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from synth import make_ground_state, random_br_vector  # noqa: E402

SAMPLED_K = (0, 7, 15)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@functools.lru_cache(maxsize=None)
def c2_state():
    return make_ground_state("C2", solver="random")


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_2203_01120_gb300 import Context, build
    build()
    c = Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def qslot(ctx):
    return ctx.load_ground_state(c2_state())


def apply_gpu(torch, ctx, q, x, mixed=False):
    from paper_2203_01120_gb300 import TDLZ_FP64, TDLZ_MIXED
    dt = torch.complex64 if mixed else torch.complex128
    xt = torch.as_tensor(x, dtype=dt, device="cuda").contiguous()
    yt = torch.zeros_like(xt)
    ctx.apply_liouvillian(q, xt, yt, False, TDLZ_MIXED if mixed else TDLZ_FP64)
    ctx.synchronize()
    return yt.cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def outputs(torch, ctx, qslot):
    gs = c2_state()
    x = random_br_vector(gs, seed=21)
    y64 = apply_gpu(torch, ctx, qslot, x)
    y32 = apply_gpu(torch, ctx, qslot, x, mixed=True)
    return x, y64, y32


@pytest.fixture(scope="module")
def oracle_sampled(outputs):
    from oracle.liouvillian import Liouvillian
    x = outputs[0]
    return Liouvillian(c2_state()).apply(x, kpoints=SAMPLED_K)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_full_size_sampled_k_fp64(outputs, oracle_sampled):
    _, y64, _ = outputs
    ks = list(SAMPLED_K)
    err = rel(y64[:, ks], oracle_sampled[:, ks])
    assert err <= 1e-12, err
    for k in ks:  # every band and side of each sampled k point, separately
        for side in range(2):
            assert rel(y64[side, k], oracle_sampled[side, k]) <= 1e-12, (k, side)


def test_full_size_sampled_k_mixed(outputs, oracle_sampled):
    _, _, y32 = outputs
    ks = list(SAMPLED_K)
    err = rel(y32[:, ks], oracle_sampled[:, ks])
    assert err <= 2e-5, err


def test_full_size_plane_stages_sampled_k(torch, ctx, outputs, oracle_sampled, monkeypatch):
    """The same operator through the fused plane stages (forced; the staged pipeline is
    the default at this size): sampled k points against the oracle, FP64 and mixed."""
    monkeypatch.setenv("TDLZ_PLANES", "1")
    q = ctx.load_ground_state(c2_state())
    x = outputs[0]
    ks = list(SAMPLED_K)
    y64 = apply_gpu(torch, ctx, q, x)
    assert rel(y64[:, ks], oracle_sampled[:, ks]) <= 1e-12
    y32 = apply_gpu(torch, ctx, q, x, mixed=True)
    assert rel(y32[:, ks], oracle_sampled[:, ks]) <= 2e-5


def test_full_size_mixed_against_fp64_everywhere(outputs):
    gs = c2_state()
    _, y64, y32 = outputs
    assert rel(y32, y64) <= 2e-5
    for k in range(gs.nk):
        assert not y64[:, k, :, :, gs.npw_kq[k]:].any()
        assert not y32[:, k, :, :, gs.npw_kq[k]:].any()


def test_full_size_pseudo_hermiticity_fp64(torch, ctx, qslot, outputs):
    """On the range of the empty-manifold projectors (where the Lanczos vectors live)
    J L is Hermitian.  a = L x and b = L x' lie in that range (L projects its
    output); then a^H J (L b) = conj(b^H J (L a))."""
    from oracle.liouvillian import jdot
    gs = c2_state()
    a = outputs[1]
    b = apply_gpu(torch, ctx, qslot, random_br_vector(gs, seed=22))
    la = apply_gpu(torch, ctx, qslot, a)
    lb = apply_gpu(torch, ctx, qslot, b)
    lhs = jdot(a, lb)            # a^H J L b
    rhs = np.conj(jdot(b, la))   # conj(b^H J L a)
    scale = np.linalg.norm(a) * np.linalg.norm(lb)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)


def test_full_size_grouped_mixed_chains(ctx, qslot):
    """Three NH chains of one q-slot in one chain set (stacked passes, graph replay
    from four steps on) against each chain alone, mixed precision, 8 steps."""
    from paper_2203_01120_gb300 import TDLZ_MIXED
    grouped = ctx.lanczos_run([qslot] * 3, [0, 1, 2], 8, "nh", TDLZ_MIXED)
    assert not np.any(grouped["status"])
    for c in range(3):
        alone = ctx.lanczos_run([qslot], [c], 8, "nh", TDLZ_MIXED)
        for key in ("alpha", "beta", "gamma", "z"):
            a, b = grouped[key][c], alone[key][0]
            assert np.max(np.abs(a - b)) <= 1e-4 * np.max(np.abs(b)), (c, key)

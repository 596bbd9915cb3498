"""GPU parity of the fused plane stages and of both real-space paths on the
CrI3-shaped grid.

The Liouvillian has two implementations of its real-space stages (chosen per
q-slot at load): the staged pipeline, which keeps every stacked vector's
real-space grids in HBM, and the fused plane stages, which transform one z plane
of one band-side at a time on chip and keep only the stick buffer in HBM (chosen
where the staged workspace would not fit, e.g. the 45x45x144, 64-k workload).
TDLZ_PLANES=1 forces the plane stages, TDLZ_PLANES=0 the staged pipeline.

Checks (tolerances as for the default path):
* one application against the oracle: FP64 <= 1e-12 (every kernel mask, the
  adjoint), mixed <= 2e-5 (tensor-core and CUDA-core contractions);
* Lanczos coefficients against the oracle, FP64, 50 steps, <= 1e-9;
* CUDA-graph replay equals eager steps bit for bit; autotuned launch shapes change
  no result; three chains grouped equal each chain alone;
* the 45x45x144 grid of the CrI3-shaped workload (hexagonal a = 13, c = 38 bohr,
  ~12000 plane waves per component; 2 of its k points and 6 bands, random
  orthonormal occupied states) through BOTH paths: every output element against
  the oracle, FP64 <= 1e-12 and mixed <= 2e-5.  This runs the 45-point x/y line
  plans and the 144 = 4 x 36 z-line plan.
"""

import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _cases import ground_state, liouvillian  # noqa: E402
from synth import make_ground_state, random_br_vector  # noqa: E402


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


def load(ctx, gs, monkeypatch, planes=True):
    monkeypatch.setenv("TDLZ_PLANES", "1" if planes else "0")
    return ctx.load_ground_state(gs)


def apply_gpu(torch, ctx, q, x, adjoint=False, mixed=False):
    from paper_2203_01120_gb300 import TDLZ_FP64, TDLZ_MIXED
    dt = torch.complex64 if mixed else torch.complex128
    xt = torch.as_tensor(x, dtype=dt, device="cuda").contiguous()
    yt = torch.zeros_like(xt)
    ctx.apply_liouvillian(q, xt, yt, adjoint, TDLZ_MIXED if mixed else TDLZ_FP64)
    ctx.synchronize()
    return yt.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,mask", [("C0", 3), ("C0K", 0), ("C0K", 1), ("C0K", 2),
                                       ("C0K", 3), ("C1", 3)])
def test_plane_stages_apply_fp64(torch, ctx, name, mask, monkeypatch):
    q = load(ctx, ground_state(name, mask), monkeypatch)
    lv = liouvillian(name, mask)
    x = random_br_vector(lv.gs, seed=7)
    y = apply_gpu(torch, ctx, q, x)
    assert rel(y, lv.apply(x)) <= 1e-12
    for k in range(lv.gs.nk):
        assert not y[:, k, :, :, lv.gs.npw_kq[k]:].any()
    ya = apply_gpu(torch, ctx, q, x, adjoint=True)
    assert rel(ya, lv.apply_adjoint(x)) <= 1e-12


@pytest.mark.parametrize("tc", ["1", "0"])
@pytest.mark.parametrize("name", ["C0K", "C1"])
def test_plane_stages_apply_mixed(torch, ctx, name, tc, monkeypatch):
    monkeypatch.setenv("TDLZ_TC", tc)
    q = load(ctx, ground_state(name), monkeypatch)
    lv = liouvillian(name)
    x = random_br_vector(lv.gs, seed=9)
    assert rel(apply_gpu(torch, ctx, q, x, mixed=True), lv.apply(x)) <= 2e-5


@pytest.mark.parametrize("flavor,mu", [("nh", 0), ("phm", 0), ("nh", 2)])
def test_plane_stages_lanczos_fp64(torch, ctx, flavor, mu, monkeypatch):
    from oracle.lanczos import run_chain
    q = load(ctx, ground_state("C1"), monkeypatch)
    got = ctx.lanczos_run([q], [mu], 50, flavor)
    ref = run_chain(liouvillian("C1"), mu, 50, flavor)
    assert got["status"][0] == 0 and got["steps_done"][0] == 50
    for key, r in (("alpha", ref.alpha), ("beta", ref.beta), ("gamma", ref.gamma)):
        assert np.max(np.abs(got[key][0] - r)) <= 1e-9 * np.max(np.abs(r)), key
    assert np.max(np.abs(got["z"][0] - ref.z)) <= 1e-9 * np.max(np.abs(ref.z))


@pytest.mark.parametrize("flavor,prec", [("nh", 1), ("phm", 0)])
def test_plane_stages_graph_replay_bitwise(torch, ctx, flavor, prec, monkeypatch):
    q = load(ctx, ground_state("C1"), monkeypatch)
    eager = ctx.chain_create([q, q], [0, 1], 13, flavor, prec)
    for _ in range(13):
        eager.advance(1)
    ref = eager.read()
    eager.close()
    g = ctx.chain_create([q, q], [0, 1], 13, flavor, prec)
    g.advance(13)
    got = g.read()
    g.close()
    for key in ("alpha", "beta", "gamma", "z", "n0", "steps_done", "status"):
        assert np.array_equal(got[key], ref[key]), key


def test_plane_stages_grouped_equal_single(torch, ctx, monkeypatch):
    q = load(ctx, ground_state("C1"), monkeypatch)
    grouped = ctx.lanczos_run([q, q, q], [0, 1, 2], 20, "nh")
    for c in range(3):
        alone = ctx.lanczos_run([q], [c], 20, "nh")
        for key in ("alpha", "beta", "gamma", "z"):
            a, b = grouped[key][c], alone[key][0]
            assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b)), (c, key)


def test_plane_stages_autotune_changes_no_result(torch, monkeypatch):
    from paper_2203_01120_gb300 import Context, TDLZ_MIXED
    lv = liouvillian("C1")
    x = random_br_vector(lv.gs, seed=31)
    out = []
    for env in ("0", "1"):
        monkeypatch.setenv("TDLZ_AUTOTUNE", env)
        c = Context(0)
        try:
            q = load(c, ground_state("C1"), monkeypatch)
            ys = [apply_gpu(torch, c, q, x), apply_gpu(torch, c, q, x, mixed=True)]
            chains = c.lanczos_run([q, q], [0, 2], 12, "nh", TDLZ_MIXED)
            report = c.autotune_report()
        finally:
            c.close()
        out.append((ys, chains, report))
    (y0, c0, r0), (y1, c1, r1) = out
    assert r0 == {} and any(k.startswith("plane_product") for k in r1), r1
    for a, b in zip(y0, y1):
        assert np.array_equal(a, b)
    for key in ("alpha", "beta", "gamma", "z"):
        assert np.array_equal(c0[key], c1[key]), key


@functools.lru_cache(maxsize=None)
def c3_small():
    return make_ground_state("C3", solver="random", kgrid=(2, 1, 1), nocc=6)


@functools.lru_cache(maxsize=None)
def c3_reference():
    from oracle.liouvillian import Liouvillian
    gs = c3_small()
    x = random_br_vector(gs, seed=41)
    return x, Liouvillian(gs).apply(x)


@pytest.mark.parametrize("planes", [False, True])
def test_c3_grid_apply_both_paths(torch, ctx, planes, monkeypatch):
    gs = c3_small()
    assert tuple(gs.fft) == (45, 45, 144)
    q = load(ctx, gs, monkeypatch, planes)
    x, ref = c3_reference()
    y64 = apply_gpu(torch, ctx, q, x)
    for side in range(2):
        for k in range(gs.nk):
            assert rel(y64[side, k], ref[side, k]) <= 1e-12, (side, k)
    assert rel(apply_gpu(torch, ctx, q, x, mixed=True), ref) <= 2e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_staged_sub_batches_change_no_result(torch, monkeypatch, prec):
    """The staged pipeline runs its real-space stages over sub-batches of the stacked
    vectors where their grids would take too much memory (one vector at a time on the
    45x45x144 workload); TDLZ_STAGED_SUB=1 forces one vector per sub-batch on C1, and the
    grouped NH chains (6 stacked vectors per pass) must equal the unsplit run bit for bit."""
    from paper_2203_01120_gb300 import Context
    out = []
    for sub in (None, "1", "4"):
        if sub is None:
            monkeypatch.delenv("TDLZ_STAGED_SUB", raising=False)
        else:
            monkeypatch.setenv("TDLZ_STAGED_SUB", sub)
        c = Context(0)
        try:
            q = load(c, ground_state("C1"), monkeypatch, planes=False)
            out.append(c.lanczos_run([q, q, q], [0, 1, 2], 10, "nh", prec))
        finally:
            c.close()
    for other in out[1:]:
        for key in ("alpha", "beta", "gamma", "z", "n0", "steps_done", "status"):
            assert np.array_equal(out[0][key], other[key]), key


@pytest.mark.parametrize("case", ["C0K", "C1", "C3grid"])
def test_fused_yx_passes_equal_separate_passes(torch, monkeypatch, case):
    """The staged pipeline's fused Y + X line kernels (one CTA per row and chunk of z
    planes, the planes in shared memory; the default, TDLZ_YX_FUSED=0 turns it off)
    transform every line with the same plan in the same order as the separate Y and X
    passes: L x in FP64 and mixed
    precision and the Lanczos coefficients are bit for bit the same."""
    from paper_2203_01120_gb300 import Context, TDLZ_MIXED
    gs = c3_small() if case == "C3grid" else ground_state(case)
    x = random_br_vector(gs, seed=61)
    out = []
    for env in ("0", "1"):
        monkeypatch.setenv("TDLZ_YX_FUSED", env)
        c = Context(0)
        try:
            q = load(c, gs, monkeypatch, planes=False)
            ys = [apply_gpu(torch, c, q, x), apply_gpu(torch, c, q, x, mixed=True),
                  apply_gpu(torch, c, q, x, adjoint=True)]
            chains = c.lanczos_run([q, q], [0, 2], 8, "nh", TDLZ_MIXED)
        finally:
            c.close()
        out.append((ys, chains))
    (y0, c0), (y1, c1) = out
    for a, b in zip(y0, y1):
        assert np.array_equal(a, b)
    for key in ("alpha", "beta", "gamma", "z"):
        assert np.array_equal(c0[key], c1[key]), key
    if case != "C3grid":
        ref = liouvillian(case).apply(x)
        assert rel(y1[0], ref) <= 1e-12

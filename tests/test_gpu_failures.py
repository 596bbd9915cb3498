"""Failure paths on the GPU, in forms that fault, trap or hang nothing.

* A bounded mbarrier wait of the tensor-core GEMMs that "expires": the test hook
  TDLZ_TEST_INJECT_TC_TIMEOUT=1 (read at context creation) makes the next wait that
  completes report expiry, so the CTA takes its abort path with every MMA finished
  (it waits for its last commit before releasing TMEM).  The next synchronising call
  returns TDLZ_ERR_TIMEOUT; the call after it runs normally and is correct.
* Per-chain truncation: a chain set over two q-slots restored from an image whose
  second group's vectors were overwritten with NaN: the chains of that group stop
  with TDLZ_ERR_NUMERIC at their first step, the other group's chains run all their
  steps and equal an uncorrupted run.
* Rejection before any step: non-finite coefficients and non-orthonormal occupied
  states in the ground state (TDLZ_ERR_ARG, with the reason in the message).
"""

import dataclasses
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from _cases import ground_state, liouvillian  # noqa: E402
from synth import random_br_vector  # noqa: E402

TDLZ_ERR_ARG, TDLZ_ERR_NUMERIC, TDLZ_ERR_TIMEOUT = 1, 6, 7


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


def apply_mixed(torch, ctx, q, x):
    from paper_2203_01120_gb300 import TDLZ_MIXED
    xt = torch.as_tensor(x, dtype=torch.complex64, device="cuda").contiguous()
    yt = torch.zeros_like(xt)
    ctx.apply_liouvillian(q, xt, yt, False, TDLZ_MIXED)
    ctx.synchronize()
    return yt.cpu().numpy().astype(np.complex128)


def test_tensor_core_wait_expiry_reported_then_recovered(torch, monkeypatch):
    from paper_2203_01120_gb300 import Context, TdlzError
    monkeypatch.setenv("TDLZ_TEST_INJECT_TC_TIMEOUT", "1")
    monkeypatch.setenv("TDLZ_TC", "1")
    c = Context(0)
    try:
        q = c.load_ground_state(ground_state("C1"))
        lv = liouvillian("C1")
        x = random_br_vector(lv.gs, seed=51)
        with pytest.raises(TdlzError) as e:
            apply_mixed(torch, c, q, x)
        assert e.value.status == TDLZ_ERR_TIMEOUT
        y = apply_mixed(torch, c, q, x)  # the injection is spent: a normal, correct call
        ref = lv.apply(x)
        assert np.linalg.norm(y - ref) <= 2e-5 * np.linalg.norm(ref)
    finally:
        c.close()


def _group_offsets(image, nchain, ngroup):
    """Byte offset of each group's vector slots in a restart image (header: 8-byte magic
    and seven ints; then (q-slot, mu) per chain and the step of each group)."""
    return struct.calcsize("8s7i") + 8 * nchain + 4 * ngroup


def test_non_finite_chain_stops_alone(torch, ctx):
    from paper_2203_01120_gb300 import TDLZ_FP64
    from synth import make_ground_state
    q1 = ctx.load_ground_state(ground_state("C0K"))
    q2 = ctx.load_ground_state(make_ground_state("C0K", q_2pi_a=(0.2, 0.0, 0.0)))
    slots, mus = [q1, q2, q1, q2], [0, 0, 2, 2]
    clean = ctx.lanczos_run(slots, mus, 12, "nh", TDLZ_FP64)
    a = ctx.chain_create(slots, mus, 6, "nh", TDLZ_FP64)
    a.advance(6)
    image = bytearray(a.save())
    a.close()
    # groups are the two q-slots in order of first appearance, each holding its chains'
    # stacked vectors (3 slots of nv vectors for NH); overwrite group 1's with NaN
    gs0, gs1 = ground_state("C0K"), make_ground_state("C0K", q_2pi_a=(0.2, 0.0, 0.0))
    br0 = 2 * gs0.nk * gs0.nocc * 2 * gs0.npwx
    br1 = 2 * gs1.nk * gs1.nocc * 2 * gs1.npwx
    nv = 2 * 2  # two NH chains per group, q and J p each
    off = _group_offsets(image, 4, 2) + 3 * nv * br0 * 16
    nan = np.full(3 * nv * br1 * 2, np.nan).tobytes()
    image[off:off + len(nan)] = nan
    b = ctx.chain_create(slots, mus, 12, "nh", TDLZ_FP64)
    b.restore(bytes(image))
    b.advance(6)
    got = b.read()
    b.close()
    for c in (1, 3):  # q-slot 2: stopped at its first step after the restart
        assert got["status"][c] == TDLZ_ERR_NUMERIC
        assert got["steps_done"][c] == 6
    for c in (0, 2):  # q-slot 1: unaffected
        assert got["status"][c] == 0 and got["steps_done"][c] == 12
        for key in ("alpha", "beta", "gamma", "z"):
            assert np.array_equal(got[key][c], clean[key][c]), (c, key)


def test_non_finite_ground_state_rejected(torch, ctx):
    from paper_2203_01120_gb300 import TdlzError
    gs = ground_state("C0")
    ck = gs.coeff_k.copy()
    ck[0, 0, 0, 0, 0] = np.nan
    with pytest.raises(TdlzError) as e:
        ctx.load_ground_state(dataclasses.replace(gs, coeff_k=ck))
    assert e.value.status == TDLZ_ERR_ARG and "non-finite" in str(e.value)


def test_non_orthonormal_occupied_states_rejected(torch, ctx):
    from paper_2203_01120_gb300 import TdlzError
    gs = ground_state("C0")
    ckq = gs.coeff_kq.copy()
    ckq[1, 0, 2] *= 1.01  # one band of the Y side at k+q no longer normalised
    with pytest.raises(TdlzError) as e:
        ctx.load_ground_state(dataclasses.replace(gs, coeff_kq=ckq))
    assert e.value.status == TDLZ_ERR_ARG and "orthonormal" in str(e.value)


def test_mixed_only_slot_refuses_fp64(torch, ctx, monkeypatch):
    """A q-slot loaded with TDLZ_MIXED_ONLY=1 (FP64 real-space orbitals released after
    the FP32 ones are built) applies L in mixed precision as before and refuses FP64
    (TDLZ_ERR_STATE) instead of reading freed data."""
    from paper_2203_01120_gb300 import TDLZ_FP64, TdlzError
    monkeypatch.setenv("TDLZ_MIXED_ONLY", "1")
    q = ctx.load_ground_state(ground_state("C1"))
    lv = liouvillian("C1")
    x = random_br_vector(lv.gs, seed=52)
    y = apply_mixed(torch, ctx, q, x)
    ref = lv.apply(x)
    assert np.linalg.norm(y - ref) <= 2e-5 * np.linalg.norm(ref)
    xt = torch.as_tensor(x, device="cuda")
    with pytest.raises(TdlzError) as e:
        ctx.apply_liouvillian(q, xt, torch.zeros_like(xt), False, TDLZ_FP64)
    assert e.value.status == 2

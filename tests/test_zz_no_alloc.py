"""tdlz_spectrum_noalloc (the allocation-free spectrum entry point) through the C ABI.

It serves callers that cannot allocate device memory themselves (their device
memory is owned by another allocator, or cudaMalloc's device-wide
synchronisation is not affordable where they call it).  Its result must equal
the allocating tdlz_spectrum's, on two calls in a row (the static scratch is
shared and reused), and sizes beyond the static scratch must be refused.
This file is collected last so that a failure here leaves every other test run.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_01120_gb300 import Context, build
    from synth import make_ground_state
    build()
    ctx = Context(0)
    q = ctx.load_ground_state(make_ground_state("C1"))
    coeffs = ctx.lanczos_run([q, q], [0, 2], 40, "nh")
    yield torch, ctx, coeffs
    ctx.close()


def _to_device(torch, coeffs):
    return {k: torch.as_tensor(np.ascontiguousarray(v), device="cuda") for k, v in coeffs.items()}


def test_noalloc_matches_allocating_entry_point(setup):
    torch, ctx, coeffs = setup
    grid = (0.0, 2000.0, 0.5, 10.0, 1)  # start, end, step, eta (meV), units
    ref = ctx.spectrum(coeffs, *grid)
    nw = ctx.spectrum_nomega(grid[0], grid[1], grid[2], grid[4])
    assert nw == ref.shape[-1]
    dev = _to_device(torch, coeffs)
    for call in range(2):
        chi = torch.full((2, 3, nw), float("nan"), dtype=torch.complex128, device="cuda")
        ctx.spectrum_noalloc(dev, *grid, chi)
        ctx.synchronize()
        got = chi.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 1e-12, (call, err)


def test_noalloc_matches_across_frequency_chunks(setup):
    """Coefficient arrays padded to 20000 steps (40 computed): the scratch then holds
    only 13 frequencies per chunk, so the 4001-point grid runs in many chunks, the
    last one shorter; every chunk must equal the allocating entry point."""
    torch, ctx, coeffs = setup
    cap = 20000
    padded = dict(coeffs)
    for key in ("alpha", "beta", "gamma"):
        a = np.zeros((2, cap), dtype=coeffs[key].dtype)
        a[:, :coeffs[key].shape[1]] = coeffs[key]
        padded[key] = a
    zpad = np.zeros((2, 3, cap), dtype=coeffs["z"].dtype)
    zpad[:, :, :coeffs["z"].shape[2]] = coeffs["z"]
    padded["z"] = zpad
    grid = (0.0, 2000.0, 0.5, 10.0, 1)
    ref = ctx.spectrum(padded, *grid)
    nw = ref.shape[-1]
    assert (32 * 2 ** 20 // 16) // (4 * cap * 2) < nw  # several chunks
    dev = _to_device(torch, padded)
    chi = torch.full((2, 3, nw), float("nan"), dtype=torch.complex128, device="cuda")
    ctx.spectrum_noalloc(dev, *grid, chi)
    ctx.synchronize()
    got = chi.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_noalloc_allocates_nothing(setup):
    """A call recorded in a CUDA graph in global capture mode (any allocation or
    synchronisation inside it would invalidate the capture) and replayed gives the
    same chi as an eager call."""
    torch, ctx0, coeffs = setup
    from paper_2203_01120_gb300 import Context
    stream = torch.cuda.Stream()
    ctx = Context(0, stream=stream.cuda_stream)
    try:
        grid = (0.0, 2000.0, 0.5, 10.0, 1)
        ref = ctx0.spectrum(coeffs, *grid)
        nw = ref.shape[-1]
        dev = _to_device(torch, coeffs)
        chi = torch.zeros((2, 3, nw), dtype=torch.complex128, device="cuda")
        ctx.spectrum_noalloc(dev, *grid, chi)  # first call on the device: before capture
        ctx.synchronize()
        chi.zero_()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="global"):
            ctx.spectrum_noalloc(dev, *grid, chi)
        g.replay()
        torch.cuda.synchronize()
        got = chi.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    torch, ctx, coeffs = setup
    from paper_2203_01120_gb300 import TdlzError
    limit = 32 * 2 ** 20 // 64  # nchain * nsteps the 32 MiB scratch can hold
    nsteps = limit + 1
    dev = {
        "steps_done": torch.ones(1, dtype=torch.int32, device="cuda"),
        "alpha": torch.zeros((1, nsteps), dtype=torch.complex128, device="cuda"),
        "beta": torch.zeros((1, nsteps), dtype=torch.float64, device="cuda"),
        "gamma": torch.zeros((1, nsteps), dtype=torch.complex128, device="cuda"),
        "z": torch.zeros((1, 3, nsteps), dtype=torch.complex128, device="cuda"),
        "n0": torch.ones(1, dtype=torch.float64, device="cuda"),
        "wk": torch.ones(1, dtype=torch.float64, device="cuda"),
    }
    chi = torch.zeros((1, 3, 11), dtype=torch.complex128, device="cuda")
    with pytest.raises(TdlzError) as e:
        ctx.spectrum_noalloc(dev, 0.0, 10.0, 1.0, 1.0, 1, chi)
    assert e.value.status == 1 and "static scratch" in str(e.value)

"""The C-ABI library builds, loads and exports every entry point declared in
include/tdlz.h; without a GPU its first call fails with TDLZ_ERR_CUDA instead of
falling back to anything (CPU only, no compute)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tdlz.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tdlz_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_01120_gb300 import build_ext
    path = build_ext.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "tdlz_apply_liouvillian" in names and "tdlz_spectrum" in names
    for n in ("tdlz_load_ground_state", "tdlz_lanczos_run", "tdlz_chain_create",
              "tdlz_chain_advance", "tdlz_chain_read", "tdlz_create", "tdlz_last_error"):
        assert n in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2203_01120_gb300 import binding
    assert set(declared_functions()) == set(binding.EXPORTS)


def test_no_gpu_means_error_not_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.tdlz_create.restype = ctypes.c_int
    st = lib.tdlz_create(ctypes.byref(h), 0, None)
    assert st == 3 and not h.value  # TDLZ_ERR_CUDA


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2203_01120_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_autotune_report_parsing():
    from paper_2203_01120_gb300.binding import parse_autotune_report
    text = ("density/f32/nr=124416/rows=2560/nvec=6=3 (1.7012 ms)\n"
            "inv_x/f32/n=36/lines=3456/rows=15360=256 (1.5590 ms)\n")
    got = parse_autotune_report(text)
    assert got == {"density/f32/nr=124416/rows=2560/nvec=6": (3, 1.7012),
                   "inv_x/f32/n=36/lines=3456/rows=15360": (256, 1.559)}
    assert parse_autotune_report("") == {}

"""NVTX ranges on the host side of the library: every stage of a Liouvillian pass, the
ground-state load and a chain's advance, graph capture and graph replay push a named
range (what an attached profiler shows on its timeline).  The injection library
tests/nvtx_log_injection.c, built here with the C compiler, logs every pushed name in a
child process (NVTX reads its injection path once per process)."""

import os
import shutil
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    sys.path.insert(0, {tests!r})
    from paper_2203_01120_gb300 import Context, TDLZ_MIXED
    from _cases import ground_state
    c = Context(0)
    q = c.load_ground_state(ground_state("C1"))
    r = c.lanczos_run([q], [0], 8, "nh", TDLZ_MIXED)
    assert r["steps_done"][0] == 8
    c.close()
""")

STAGES = ("scatter", "fft_inv", "density", "hartree", "potential", "product", "fft_fwd",
          "gather", "vnl", "pc", "lanczos")


def test_stage_ranges_pushed(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_01120_gb300 import build_ext
    build_ext.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler for the injection library")
    inc = os.path.join(os.path.dirname(os.path.dirname(build_ext.nvcc())), "include")
    so = str(tmp_path / "nvtx_log_injection.so")
    subprocess.run([cc, "-shared", "-fPIC", "-O2", "-I", inc,
                    os.path.join(HERE, "nvtx_log_injection.c"), "-o", so], check=True)
    log = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=so, TDLZ_TEST_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, tests=HERE)], env=env,
                   check=True, timeout=900)
    names = set(log.read_text().split())
    missing = [s for s in STAGES if f"tdlz/{s}" not in names]
    assert not missing, (missing, sorted(names))
    for r in ("tdlz/load_ground_state", "tdlz/advance", "tdlz/capture", "tdlz/graph_replay"):
        assert r in names, (r, sorted(names))

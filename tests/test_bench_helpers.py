"""Host-side helpers of the benchmark line (no GPU): the FP64 roofline object, the
whole-job rate of the replicas, the workload label and the ncu traffic lookup."""

import math

import bench


def test_fp64_roofline_is_flops_over_event_time():
    prof = {"fft_inv": {"ms": 300.0, "flops": 2.4e11, "launches": 4, "bytes": 1.0},
            "density": {"ms": 100.0, "flops": 0.6e11, "launches": 2, "bytes": 1.0},
            "hartree": {"ms": 0.0, "flops": 0.0, "launches": 0, "bytes": 0.0}}
    r = bench.fp64_roofline(prof)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["achieved"], 3.0e11 / 0.4 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / bench.FP64_PEAK_TFLOPS)
    assert bench.fp64_roofline({}) is None


def test_whole_job_rate_counts_every_rank_against_the_slowest():
    # 4 replicas of 3 chains, 20 steps, slowest rank 0.5 s
    assert math.isclose(bench.whole_job_rate(4, 3, 20, 0.5), 4 * 3 * 20 / 0.5)


def test_workload_label_follows_the_config():
    assert bench.workload("C2") == bench.WORKLOAD
    w = bench.workload("C1")
    assert w.startswith("C1:") and "FFT 16x16x16" in w and "Nocc=8" in w


class _Args:
    def __init__(self, **kw):
        self.kpoints, self.flavor, self.chains, self.config = 0, "nh", 3, "C2"
        self.__dict__.update(kw)


def test_ncu_traffic_only_for_the_captured_configuration():
    assert bench.ncu_traffic(_Args(), "product") == bench.NCU_TRAFFIC.get(("C2", "product"))
    assert bench.ncu_traffic(_Args(kpoints=4), "product") is None
    assert bench.ncu_traffic(_Args(flavor="ph"), "product") is None
    assert bench.ncu_traffic(_Args(chains=1), "product") is None
    assert bench.ncu_traffic(_Args(), "density") is None


def test_algorithmic_work_of_a_c2_step():
    """One NH step of three chains on the C2 shapes: 6V per chain + 2V of orbitals +
    the projector table (V = 2 x 16 x 40 x 2 x 5085 complex, 8 bytes each), and six
    Liouvillian applications of ~6.9e10 flop."""
    from types import SimpleNamespace
    gs = SimpleNamespace(nk=16, nocc=40, nproj=64, npw_kq=[5085] * 16, fft=(36, 36, 96))
    b, f = bench.algorithmic_work(gs, "nh", 3, 8)
    v = 2 * 16 * 40 * 2 * 5085
    assert math.isclose(b, (18 * v + 2 * v + 16 * 64 * 5085) * 8)
    assert 2.1e9 < b < 2.15e9
    assert 4.1e11 < f < 4.2e11
    bp, fp = bench.algorithmic_work(gs, "ph", 3, 8)
    assert math.isclose(fp, f / 2) and bp < b


def test_chi_column_errors_normalise_by_the_diagonal():
    import numpy as np
    ref = np.ones((3, 3, 5), dtype=complex)
    ref[0, 1] *= 1e-6  # a tiny off-diagonal component
    got = ref.copy()
    got[0, 1] += 1e-3
    e = bench.chi_column_errors(got, ref)
    assert math.isclose(e[0], 1e-3 * math.sqrt(5) / math.sqrt(5)) and e[1] == 0 and e[2] == 0


def test_sphere_sticks_and_planes_count_distinct_columns():
    import numpy as np
    from types import SimpleNamespace
    mil = np.array([[[0, 0, 0], [0, 0, 1], [1, 0, 0], [1, 2, 5], [0, 0, 0]]], dtype=np.int32)
    gs = SimpleNamespace(nk=1, miller_kq=mil, npw_kq=np.array([4]))
    assert bench.sphere_sticks_planes(gs) == (3, 2)

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

"""Host-side logic of bench.py (no GPU): relaxation times of the workloads, algorithmic bytes, the
mirror of the library's automatic kernel choice used to name the roofline kernel, the rule under
which a recorded ncu traffic figure is reported, and the parsing of the clock samples."""
import os

import pytest

import bench


def test_tau_of_the_workloads():
    # tau = 3 u N / Re + 1/2 (lattice viscosity nu = u N / Re = (tau - 1/2) / 3)
    assert bench.tau_of(bench.WORKLOADS["d3q19_256_fp32_re1000"]) == pytest.approx(0.5768)
    assert bench.tau_of(bench.WORKLOADS["d2q9_128_fp64_re100"]) == pytest.approx(0.884)
    assert bench.tau_of(bench.WORKLOADS["d3q19_512_fp32_re1000"]) == pytest.approx(0.6536)


def test_algorithmic_bytes_per_cell():
    # q populations read + q written
    assert bench.algorithmic_bytes_per_cell(bench.WORKLOADS["d3q19_256_fp32_re1000"]) == 152
    assert bench.algorithmic_bytes_per_cell(bench.WORKLOADS["d3q19_512_f16s_re1000"]) == 76
    assert bench.algorithmic_bytes_per_cell(bench.WORKLOADS["d2q9_128_fp64_re100"]) == 144
    assert bench.algorithmic_bytes_per_cell(bench.WORKLOADS["d2q9_1024_learned"]) == 72


@pytest.mark.parametrize("workload,kernel", [
    ("d3q19_256_fp32_re1000", "fused_step_kernel"),       # FP32 D3Q19: one cell per thread
    ("d3q19_512_fp32_re1000", "fused_step_kernel"),
    ("d3q19_512_f16s_re1000", "fused_step_pair_kernel"),  # 16-bit storage: two cells
    ("d3q19_512_bf16s_re1000", "fused_step_pair_kernel"),
    ("d2q9_128_fp64_re100", "fused_step_kernel"),         # FP64: one cell
    ("d2q9_1024_learned", "fused_step_pair_kernel"),      # FP32 D2Q9 >= 2^17 cells: two cells
])
def test_step_kernel_of_the_automatic_choice(workload, kernel):
    assert bench.step_kernel_of(bench.WORKLOADS[workload])[0] == kernel


def test_step_kernel_of_small_and_forced():
    w = dict(bench.WORKLOADS["d2q9_1024_learned"])
    w["n"] = 256  # 2^16 cells: below the two-cell threshold for FP32 D2Q9
    assert bench.step_kernel_of(w)[0] == "fused_step_kernel"
    w["n"] = 384
    assert bench.step_kernel_of(w)[0] == "fused_step_pair_kernel"
    w["n"] = 385  # odd nx: the two-cell kernel does not apply
    assert bench.step_kernel_of(w)[0] == "fused_step_kernel"
    d = bench.WORKLOADS["d3q19_256_fp32_re1000"]
    assert bench.step_kernel_of(d, "pair")[0] == "fused_step_pair_kernel"
    assert bench.step_kernel_of(d, "tma")[0] == "fused_step_tma_kernel"
    assert bench.step_kernel_of(d, "cell")[0] == "fused_step_kernel"
    for name in bench.step_kernel_of(d, "tma")[1]:
        assert os.path.exists(os.path.join(bench.ROOT, "paper_1507_06767_gb300", "csrc", name))


def test_recorded_traffic_only_for_the_profiled_kernel_and_size():
    wl = "d3q19_256_fp32_re1000"
    w = dict(bench.WORKLOADS[wl])
    assert bench.recorded_traffic(wl, w, "pair") is None
    assert bench.recorded_traffic(wl, w, "cell") is None
    small = dict(w, n=128)
    assert bench.recorded_traffic(wl, small) is None
    got = bench.recorded_traffic(wl, w)
    path = os.path.join(bench.ROOT, "profiles", f"fused_step_{wl}.md")
    txt = open(path).read()
    if f"kernel_source_sha256_16: {bench.kernel_source_hash(w)}" in txt:
        assert got is not None and 0.9 * 2 * 19 * 4 * 256 ** 3 < got < 1.1 * 2 * 19 * 4 * 256 ** 3
    else:
        assert got is None
    assert bench.recorded_traffic("d2q9_1024_learned", bench.WORKLOADS["d2q9_1024_learned"]) is None


def test_recorded_cycle_traffic_only_for_the_profiled_schedule():
    wl = "d3q19_blocks_512_3level"
    w = dict(bench.WORKLOADS[wl])
    assert bench.recorded_cycle_traffic(wl, dict(w, n=256)) is None
    assert bench.recorded_cycle_traffic(wl, w, persistent=True) is None
    assert bench.recorded_cycle_traffic(wl, w, fusion="separate") is None
    assert bench.recorded_cycle_traffic(wl, w, step_form="pair") is None
    got = bench.recorded_cycle_traffic(wl, w)
    path = os.path.join(bench.ROOT, "profiles", f"cycle_dram_{wl}.md")
    txt = open(path).read() if os.path.exists(path) else ""
    if f"kernel_source_sha256_16: {bench.cycle_source_hash()}" in txt:
        # at least the algorithmic 152 B per cell update of the 57.7 M updates of a cycle, less
        # what stays in L2 between launches, and not more than twice that
        assert got is not None and 0.8 * 152 * 57671680 < got < 2.0 * 152 * 57671680
    else:
        assert got is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _stamp(sec):
    import datetime

    return datetime.datetime.fromtimestamp(sec).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


def test_clock_sampler_parses_and_filters_samples():
    s = bench.ClockSampler("GPU-a")
    s.proc, s.thread = _Proc(), _Thread()
    t = 1_800_000_000.0
    s.lines = [
        f"{_stamp(t)}, GPU-a, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        f"{_stamp(t + 1)}, GPU-a, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        # another GPU
        f"{_stamp(t + 1)}, GPU-b, 900, 2070, 100.0, 0x8, Active, Not Active, Not Active, Not Active",
        f"{_stamp(t + 2)}, GPU-a, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        f"{_stamp(t + 3)}, GPU-a, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    c = s.stop()  # no timed window marked: every sample counts
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["samples"] == 3 and c["samples_under_load"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert c["sm_mhz_bins"] == {"2070": 2, "1980": 1}
    assert c["power_w_max"] == 1390.0

    # only the samples inside a timed window count as under load
    s.window(t + 0.5, t + 1.5)
    c = s.stop()
    assert c["samples"] == 3 and c["samples_under_load"] == 1
    assert c["sm_mhz"] == 1980.0 and c["reasons"] == ["sw_power_cap"]
    assert c["sm_mhz_bins"] == {"1980": 1}


def test_clock_sampler_without_samples():
    s = bench.ClockSampler(None)
    assert s.stop() is None  # never started
    s.proc, s.thread, s.lines = _Proc(), _Thread(), []
    assert s.stop() is None

"""Host logic of bench.py on CPU: the nvidia-smi clock samples it reports
beside the bench line, and the ncu DRAM traffic it reports only while the
step kernels' sources are the ones the counters were taken on."""
import bench


class _Proc:  # stands for the nvidia-smi sampling process
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc, s.thread, s.lines = _Proc(), _Thread(), list(lines)
    return s


def test_clock_samples_median_and_reasons():
    na = "Not Active"
    r = _sampler([
        f"0, 2070, 2070, 900.5, 0x0000000000000000, {na}, {na}, {na}, {na}",
        f"0, 2055, 2070, 1390.0, 0x0000000000000004, {na}, {na}, {na}, Active",
        f"0, 1980, 2070, 1399.0, 0x0000000000000004, {na}, {na}, {na}, Active",
        "not a sample",
    ]).stop()
    assert r["sm_mhz"] == 2055.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_samples_flag_thermal_and_hw_slowdown():
    na = "Not Active"
    r = _sampler([
        f"0, 1500, 2070, 1000.0, 0x48, Active, {na}, Active, {na}",
        f"0, 1600, 2070, 1000.0, 0x48, {na}, Active, {na}, {na}",
    ]).stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1550.0


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_only_for_the_sources_it_was_taken_on(monkeypatch):
    cells = 128 * 128 * 512
    for form in ("fp32", "fp16", "reduced"):
        rec = bench.TRAFFIC[("rt3d", form)]
        monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["sources"])
        assert bench.traffic_per_launch("rt3d", form, cells) == rec["bytes_per_cell"] * cells
        monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed source")
        assert bench.traffic_per_launch("rt3d", form, cells) is None
    assert bench.traffic_per_launch("rt2d", "fp32", 64 * 256) is None  # never captured


def test_kernel_source_hash_is_stable():
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16

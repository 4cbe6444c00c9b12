"""Host logic of bench.py that needs no GPU: the clock sampler keeps only the samples taken
inside the timed region and reports the throttle reasons seen there; the profile lookup
reuses recorded DRAM bytes only for the kernel code they were captured from."""
import os

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler()
    s.nvml.ok = False  # the nvidia-smi path
    s.proc = _Proc()
    s.lines = lines
    return s


class _FakeNvml:
    ok = True
    max_mhz = 2070.0


def test_nvml_samples_windowed_to_the_timed_region():
    """The NVML poller's samples (host time, MHz, reasons) are windowed like nvidia-smi's."""
    s = bench.ClockSampler()
    s.nvml = _FakeNvml()
    s.t = __import__("threading").Thread(target=lambda: None)
    s.t.start()
    s.samples = [(0.5, 1200.0, ["hw_slowdown"]), (1.01, 2070.0, []), (1.02, 2070.0, ["sw_power_cap"]),
                 (1.03, 2055.0, []), (2.5, 900.0, ["sw_thermal_slowdown"])]
    clk = s.stop(1.0, 2.0)
    assert clk["samples"] == 3 and clk["during_timed_region"] and clk["sm_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"] and clk["sm_max_mhz"] == 2070.0


def _line(sm, reasons=("Not Active",) * 4):
    return f"{sm}, 2070, 900.0, 0x0, " + ", ".join(reasons)


def test_clock_samples_outside_the_timed_region_are_ignored():
    lines = [(0.5, _line(1200, ("Active", "Not Active", "Not Active", "Not Active"))),
             (1.1, _line(2070)), (1.2, _line(2055)), (1.3, _line(2070)),
             (2.5, _line(900, ("Not Active", "Not Active", "Not Active", "Active")))]
    clk = _sampler(lines).stop(1.0, 2.0)
    assert clk["samples"] == 3 and clk["during_timed_region"]
    assert clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == []


def test_clock_throttle_inside_the_region_is_reported():
    lines = [(1.1, _line(1500, ("Not Active", "Not Active", "Active", "Not Active"))), (1.2, _line(2070))]
    clk = _sampler(lines).stop(1.0, 2.0)
    assert clk["reasons"] == ["sw_thermal_slowdown"]


def test_clock_falls_back_to_all_samples_when_none_fell_inside():
    clk = _sampler([(0.5, _line(2070)), (3.0, _line(2040))]).stop(1.0, 1.001)
    assert clk["samples"] == 2 and not clk["during_timed_region"]


def test_profiled_traffic_requires_the_recorded_code_hash(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    body = "dram_bytes_per_launch: 1000\nunits: 10\nsource_sha: {}\n"
    (tmp_path / "profiles" / "raster_bwd_replica_x.md").write_text(body.format(bench.kernel_source_sha()))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # kernel_source_sha reads the sources under ROOT: keep them reachable
    for f in bench.KERNEL_SOURCES:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_text(open(os.path.join(os.path.dirname(bench.__file__), f)).read())
    assert bench.profiled_traffic("raster_bwd", 20) == 2000.0   # scaled by the units processed
    (tmp_path / "profiles" / "raster_bwd_replica_x.md").write_text(body.format("0000000000000000"))
    assert bench.profiled_traffic("raster_bwd", 20) is None


def test_code_hash_ignores_comments():
    a = "int f() { return 1; }  // one\n/* block\n comment */\nint g;\n"
    b = "// header\nint f() { return 1; }\n\nint g;   \n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("return 1", "return 2"))

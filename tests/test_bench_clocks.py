"""The benchmark's clock record (CPU only): the summary of NVML samples and of
nvidia-smi lines gives the median SM clock, the maximum clock and every
throttle reason that was active in any sample, the ones the timing rules
reject included (hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown)."""
import bench


def test_nvml_samples_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.samples = [(2070, 2070, 0), (2055, 2070, 0x4), (2070, 2070, 0), (1980, 2070, 0x40 | 0x1)]
    out = s.summary()
    assert out["sm_mhz"] == 2062.5 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["samples"] == 4 and out["source"].startswith("nvml")


def test_nvml_reason_bits_are_the_rejected_and_noted_ones():
    names = set(bench.ClockSampler.NVML_REASONS.values())
    assert names == {"sw_power_cap", "hw_slowdown", "sw_thermal_slowdown", "hw_thermal_slowdown"}
    s = bench.ClockSampler(0)
    s.samples = [(2070, 2070, 0x8), (2070, 2070, 0x20)]
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_nvidia_smi_lines_and_the_unsampled_case():
    s = bench.ClockSampler(0)
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
               "garbage"]
    out = s.summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 2
    assert bench.ClockSampler(0).summary() == {"sm_mhz": None, "sm_max_mhz": None,
                                                "reasons": ["unsampled"], "samples": 0}

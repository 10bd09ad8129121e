"""The benchmark's clock record (host logic, no GPU): samples are kept only when nvidia-smi's own
timestamp lies inside the timed region, and throttle reasons are read from the right columns."""
import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return [ts, "0", str(sm), "2070", "900.5", "0x0000000000000000", *reasons]


def test_only_samples_inside_the_region_count():
    t0 = 1_800_000_000.0
    rows = [_row(t0 - 0.3, 1200), _row(t0 + 0.02, 2070), _row(t0 + 0.05, 2055),
            _row(t0 + 0.08, 2070, ("Not Active", "Not Active", "Not Active", "Active")), _row(t0 + 0.4, 900)]
    out = bench.ClockSampler.summarize(rows, t0, t0 + 0.1)
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["region_s"] == 0.1 and "note" not in out


def test_fallbacks_without_a_region_or_without_samples_inside_it():
    t0 = 1_800_000_000.0
    rows = [_row(t0, 2070, ("Active", "Not Active", "Not Active", "Not Active")), _row(t0 + 0.5, 1800),
            ["garbage"], ["2026/12/03 bad", "0", "x"]]
    out = bench.ClockSampler.summarize(rows)
    assert out["samples"] == 2 and out["sm_mhz"] == (2070.0 + 1800.0) / 2 and out["reasons"] == ["hw_slowdown"]
    near = bench.ClockSampler.summarize(rows, t0 + 0.05, t0 + 0.2)       # nothing inside: the sample 0.05 s away
    assert near["samples"] == 1 and near["sm_mhz"] == 2070.0 and "within 0.1 s" in near["note"]
    far = bench.ClockSampler.summarize(rows, t0 + 5.0, t0 + 6.0)
    assert far["samples"] == 2 and "all samples" in far["note"]
    no_ts = [["?", *r[1:]] for r in rows if len(r) == 10]
    assert "unreadable" in bench.ClockSampler.summarize(no_ts, t0, t0 + 1.0)["note"]


def test_smi_id_names_the_cuda_device_not_its_ordinal():
    # the UUID wins over everything, with or without its "GPU-" prefix
    assert bench.smi_gpu_id(0, "5f0b1c2d-aaaa-bbbb-cccc-0123456789ab", "3") == "GPU-5f0b1c2d-aaaa-bbbb-cccc-0123456789ab"
    assert bench.smi_gpu_id(0, "GPU-abc", None) == "GPU-abc"
    assert bench.smi_gpu_id(0, "MIG-abc", None) == "MIG-abc"
    # without a UUID: the ordinal's entry of CUDA_VISIBLE_DEVICES (an nvidia-smi index or a UUID)
    assert bench.smi_gpu_id(0, None, "3") == "3"
    assert bench.smi_gpu_id(1, None, "5, 2") == "2"
    assert bench.smi_gpu_id(0, None, "GPU-1234") == "GPU-1234"
    # only with no mapping at all is the ordinal used
    assert bench.smi_gpu_id(2, None, None) == "2"
    assert bench.smi_gpu_id(4, None, "1,2") == "4"

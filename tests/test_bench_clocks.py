"""Host logic of the bench's clock record: nvidia-smi CSV rows are parsed into the
median SM clock, the maximum clock and the throttle reasons seen, and the rows
taken before the timed region started are left out (when later rows exist)."""
import os
import tempfile

import bench


def _sampler(lines, skip):
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.skip = skip
    return s


ROW = "{sm}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}"


def test_rows_before_the_timed_region_are_dropped():
    s = _sampler([ROW.format(sm=1200, cap="Not Active"), ROW.format(sm=2070, cap="Not Active"),
                  ROW.format(sm=2040, cap="Active"), ROW.format(sm=2070, cap="Not Active")], skip=1)
    c = s.summary()
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(s.path)


def test_only_early_rows_are_kept_rather_than_none():
    c = _sampler([ROW.format(sm=2070, cap="Not Active")], skip=1).summary()
    assert c["samples"] == 1 and c["sm_mhz"] == 2070.0 and c["reasons"] == []


def test_no_sampler_process_gives_no_record():
    s = bench.ClockSampler(0)
    assert s.summary() is None

"""Host-side pieces of bench.py that need no GPU: the clock record taken during the timed
region (median SM clock, the largest maximum clock, and every throttle reason seen), and the
workload's problem list."""
import bench


class _FakeSmi:
    """Stands in for the nvidia-smi process: its CSV lines as they would be printed."""

    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _line(sm, mx, reasons=("Not Active",) * 4):
    return f"0, {sm}, {mx}, 900.1, 0x0, " + ", ".join(reasons)


def test_clock_record_median_max_and_reasons():
    s = bench.ClockSampler(0)
    lines = [_line(2070, 2070), _line(2070, 2070), _line(1980, 2070),
             _line(2070, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
             "garbage line", "0, [N/A], 2070, 1.0, 0x0, a, b, c, d"]
    s.proc = _FakeSmi("\n".join(lines) + "\n")
    rec = s.stop()
    assert rec["samples"] == 4
    assert rec["sm_mhz"] == 2070.0
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_reports_slowdowns():
    s = bench.ClockSampler(0)
    s.proc = _FakeSmi("\n".join([_line(1500, 2070, ("Active", "Not Active", "Active", "Not Active")),
                                 _line(1400, 2070)]))
    rec = s.stop()
    assert rec["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1450.0


def test_clock_record_without_samples_is_none():
    s = bench.ClockSampler(0)
    assert s.stop() is None                      # never started
    s.proc = _FakeSmi("")
    assert s.stop() is None


def test_workload_is_the_six_3d_problems():
    probs = bench.problems(6)
    assert [(p.n, p.d) for p in probs] == [(255, 3)] * 6
    assert sorted({p.alpha for p in probs}) == [0.25, 0.5, 0.75]
    assert sorted({p.gamma for p in probs}) == [1e-3, 1e-1]
    assert len({(p.alpha, p.gamma) for p in probs}) == 6
    assert all(p.beta == 1.0 for p in probs)

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


def test_workload_is_the_mixed_batch():
    """The batching form's 512 problems: every grid class, alpha in [0.1, 0.9], gamma in
    [1e-4, 1], rank 1-8 Gaussian right-hand sides, the 1e-6 settings."""
    probs = bench.problems(512)
    assert len(probs) == 512 and all(p.d == 3 and p.beta == 1.0 for p in probs)
    assert {p.n for p in probs} == {127, 255, 511, 1023, 2047}
    assert all(0.1 <= p.alpha <= 0.9 and 1e-4 <= p.gamma <= 1.0 for p in probs)
    assert all(1 <= len(p.rhs()[0]) <= 8 for p in probs)
    assert all((p.tol, p.eps, p.max_rank, p.max_tucker) == (1e-7, 1e-8, 256, 56) for p in probs)
    ref = bench.reference_problem(probs)
    assert ref.n == 127 and len(ref.rhs()[0]) == min(len(p.rhs()[0]) for p in probs if p.n == 127)


def test_arguments_and_peaks():
    a = bench.parse(["--steps", "4", "--warmup", "3", "--batch", "64"])
    assert (a.steps, a.warmup, a.batch, a.impl) == (4, 3, 64, "ours")
    assert "3d_mixed_batch_512problems" in bench.workload_name(512)
    assert bench.workload_name(64).endswith("_step64")
    pk = bench.alu_peaks(2070.0)
    assert abs(pk["fp64_tflops"] - 1.25856) < 1e-9 and abs(pk["fp32_tflops"] - 80.54784) < 1e-6

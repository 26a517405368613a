"""The launch schedule and the autotuner's search, on the host (no GPU): the schedule's ranges,
and coordinate descent on costs whose minimum is known, through the C ABI with a Python cost
callback."""
import math

import pytest

from paper_1809_01971_gb300 import fc

FIELDS = ("gemm_cover", "gemm_split", "tc_split", "tc_min_log2", "workers", "order")
CANDIDATES = {"gemm_cover": (1, 2, 4, 8, 16), "gemm_split": (0, 1, 2, 4, 8), "tc_split": (0, 1),
              "tc_min_log2": (20, 22, 24, 26), "workers": (8, 16, 24, 32), "order": (0, 1)}
DEFAULT = dict(gemm_cover=8, gemm_split=4, tc_split=1, tc_min_log2=22, workers=16, order=0)
# evaluations of one full pass from a start on the candidate lists: every other value of
# every field
PASS = sum(len(v) - 1 for v in CANDIDATES.values())


@pytest.fixture(autouse=True)
def _restore_schedule():
    prev = fc.fc_get_schedule()
    yield
    fc.fc_set_schedule(prev)


def test_default_and_round_trip():
    assert fc.fc_get_schedule().as_dict() == DEFAULT
    fc.fc_set_schedule(gemm_cover=1, gemm_split=0, tc_split=0, tc_min_log2=40, workers=64, order=1)
    assert fc.fc_get_schedule().as_dict() == dict(gemm_cover=1, gemm_split=0, tc_split=0,
                                                 tc_min_log2=40, workers=64, order=1)


@pytest.mark.parametrize("field,bad", [("gemm_cover", 0), ("gemm_cover", 65), ("gemm_split", -1),
                                       ("gemm_split", 17), ("tc_split", 2), ("tc_min_log2", 9),
                                       ("tc_min_log2", 41), ("workers", 0), ("workers", 65),
                                       ("order", 2)])
def test_out_of_range_is_rejected_and_changes_nothing(field, bad):
    before = fc.fc_get_schedule().as_dict()
    with pytest.raises(fc.FCError) as e:
        fc.fc_set_schedule(**{field: bad})
    assert e.value.code == fc.FC_EINVAL
    assert fc.fc_get_schedule().as_dict() == before


def _separable(opt):
    def cost(s):
        return 1.0 + sum(abs(math.log2(s[k] + 1) - math.log2(v + 1)) for k, v in opt.items())
    return cost


def test_separable_cost_reaches_its_minimum_in_one_pass():
    opt = dict(gemm_cover=2, gemm_split=1, tc_split=0, tc_min_log2=22, workers=32, order=1)
    seen = []
    cost = _separable(opt)

    def logged(s):
        seen.append(dict(s))
        return cost(s)

    best, c, n = fc.fc_autotune(logged, passes=1, min_gain=0.0)
    assert best.as_dict() == opt and c == 1.0
    assert n == len(seen) == 1 + PASS
    assert seen[0] == DEFAULT                         # the start is the process schedule
    # every candidate differs in exactly one field from the best schedule seen before it
    best_s, best_c = seen[0], cost(seen[0])
    for s in seen[1:]:
        assert sum(s[k] != best_s[k] for k in FIELDS) == 1
        if cost(s) < best_c:
            best_s, best_c = s, cost(s)
    assert fc.fc_get_schedule().as_dict() == DEFAULT  # the process schedule is not changed


def test_stops_after_a_pass_that_keeps_nothing():
    opt = dict(gemm_cover=4, gemm_split=2, tc_split=1, tc_min_log2=20, workers=8, order=0)
    best, c, n = fc.fc_autotune(_separable(opt), passes=5, min_gain=0.0)
    assert best.as_dict() == opt
    assert n == 1 + 2 * PASS                          # the second pass keeps nothing


def test_start_schedule_is_used():
    start = fc.fc_schedule(16, 8, 0, 26, 32, 1)
    seen = []
    fc.fc_autotune(lambda s: seen.append(dict(s)) or 1.0, start=start, passes=1)
    assert seen[0] == start.as_dict()


def test_min_gain_keeps_noise_out():
    """A candidate only 1 % better than the best so far is kept with min_gain 0, not with 2 %."""
    def cost(s):
        return 0.99 if s["workers"] == 24 else 1.0
    best, c, _ = fc.fc_autotune(cost, min_gain=0.02)
    assert best.workers == 16 and c == 1.0
    best, c, _ = fc.fc_autotune(cost, min_gain=0.0)
    assert best.workers == 24 and c == 0.99


@pytest.mark.parametrize("bad", [float("nan"), -1.0, float("inf"), "raise"])
def test_failed_candidates_are_never_kept(bad):
    def cost(s):
        if s["gemm_split"] == 0:
            if bad == "raise":
                raise RuntimeError("candidate failed")
            return bad
        return 1.0 + abs(s["gemm_split"] - 1)
    best, c, _ = fc.fc_autotune(cost, min_gain=0.0)
    assert best.gemm_split == 1 and c == 1.0


def test_coupled_cost_ends_where_no_single_change_helps():
    """Non-separable cost: coordinate descent ends at a point that no change of one field to
    one of its candidates improves."""
    def cost(s):
        return (1.0 + (math.log2(s["gemm_cover"]) - math.log2(s["workers"] / 4)) ** 2
                + 0.1 * abs(s["gemm_split"] - s["order"] * 4) + 0.05 * s["tc_split"]
                + 0.01 * abs(s["tc_min_log2"] - 22))
    best, c, _ = fc.fc_autotune(cost, passes=8, min_gain=0.0)
    b = best.as_dict()
    assert c == pytest.approx(cost(b))
    for k in FIELDS:
        for v in CANDIDATES[k]:
            assert cost({**b, k: v}) >= c - 1e-15


def test_bad_arguments():
    ok = lambda s: 1.0  # noqa: E731
    for kw in (dict(passes=0), dict(passes=9), dict(min_gain=1.0), dict(min_gain=-0.1)):
        with pytest.raises(fc.FCError):
            fc.fc_autotune(ok, **kw)
    with pytest.raises(fc.FCError):                   # the start itself failed
        fc.fc_autotune(lambda s: float("nan"))
    with pytest.raises(fc.FCError):                   # start out of range
        fc.fc_autotune(ok, start=fc.fc_schedule(0, 4, 1, 24, 16, 0))

"""Host-side accounting of the benchmark line (no GPU): the algorithmic work per
unit, its scaling by a trace's tallies, the issue-rate peak, and the guard that
drops ncu-derived figures once the kernel sources differ from the captured ones."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _tally(**kw):
    t = dict(emitted=0, miss=0, exit_front=0, exit_back=0, exit_side=0, collisions=0, refl_hist=[0] * 16)
    t.update(kw)
    return t


def test_per_unit_counts(bench):
    # the itemised counts per unit: emitted ray, entered ray, straight segment,
    # tentative collision, exit
    assert sum(bench.ALGO_PER_RAY.values()) == 110
    assert sum(bench.ALGO_PER_ENTERED.values()) == 104
    assert sum(bench.ALGO_PER_SEGMENT.values()) == 124
    assert sum(bench.ALGO_PER_COLLISION.values()) == 108
    assert sum(bench.ALGO_PER_EXIT.values()) == 30
    assert bench.ALGO_PER_END == 3
    # one Philox block for every ray, one more for every ray that entered, one per collision
    assert bench.ALGO_PER_RAY["philox_block"] == bench.ALGO_PER_ENTERED["philox_block"] == 40
    assert bench.ALGO_PER_COLLISION["philox_block"] == 40


def test_counts_scale_with_the_tallies(bench):
    f = bench.algorithmic_instructions
    assert f(_tally()) == 0
    # a miss: the geometric part only
    assert f(_tally(emitted=1, miss=1)) == 110
    # a ray that crosses the crystal without a collision and leaves through the back
    assert f(_tally(emitted=1, exit_back=1, refl_hist=[1] + [0] * 15)) == 110 + 104 + 124 + 30 + 3
    # one reflection (a second straight segment) after three tentative collisions
    t = _tally(emitted=1, exit_front=1, collisions=3, refl_hist=[0, 1] + [0] * 14)
    assert f(t) == 110 + 104 + 2 * 124 + 3 * 108 + 30 + 3
    # linear in the tallies
    a = _tally(emitted=5, miss=2, exit_front=2, exit_side=1, collisions=7, refl_hist=[1, 2] + [0] * 14)
    b = _tally(emitted=10, miss=4, exit_front=4, exit_side=2, collisions=14, refl_hist=[2, 4] + [0] * 14)
    assert f(b) == 2 * f(a)


def test_issue_peak_and_fraction(bench):
    t = _tally(emitted=10 ** 8, miss=6 * 10 ** 7, exit_back=4 * 10 ** 7, collisions=3 * 10 ** 7,
               refl_hist=[4 * 10 ** 7] + [0] * 15)
    achieved, peak = bench.algorithmic_roofline(t, 1e-3, 2070.0)
    # 152 SMs x 4 sub-partitions x 32 lanes x 2.07 GHz, in T lane-instructions/s
    assert peak == pytest.approx(40.27392, rel=1e-12)
    assert achieved == pytest.approx(bench.algorithmic_instructions(t) / 1e-3 / 1e12, rel=1e-12)


def test_ncu_figures_follow_the_captured_sources(bench, monkeypatch):
    # traffic and per-pipe counts are reported only for the kernel sources they were taken on
    assert bench.measured_traffic(10 ** 8) is not None or bench.sources_hash() != bench.TRAFFIC_SOURCE_HASH
    monkeypatch.setattr(bench, "TRAFFIC_SOURCE_HASH", "0" * 16)
    assert bench.measured_traffic(10 ** 8) is None

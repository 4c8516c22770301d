"""bench.py's launch schedule (which timed steps launch more than the step
kernel) on CPU: it must name the same kernels pic_step launches, which the
bench re-checks on the GPU against the library's own launch timers."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_schedule_of_the_bench_workload():
    cfg = bench.workload(2_000_000, 1236)
    ex = [bench.extra_launches(cfg, 30 + k) for k in range(3000)]
    # steps 400, 800, ..., 2800: both species compacted (3 kernels each);
    # every 40th step a TP step, and at the 50th TP step its compaction
    assert sum(ex) == 7 * 2 * 3 + 75 + 3
    assert sum(1 for x in ex if x == 0) == 3000 - 75
    assert bench.extra_launches(cfg, 399) == 2 * 3 + 1          # step 400: compactions and a TP step
    assert bench.extra_launches(cfg, 1999) == 2 * 3 + 1 + 3     # step 2000: both, TP step 50, its compaction
    assert bench.extra_launches(cfg, 400) == 0


def test_schedule_without_sputtering_or_compaction():
    cfg = bench.workload(1000, 1)
    cfg.update(sputter_enable=0, sort_every_e=0, sort_every_i=0)
    assert all(bench.extra_launches(cfg, h) == 0 for h in range(2000))

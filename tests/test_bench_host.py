"""Host-side accounting of bench.py (no GPU): the launch counts it reports
follow the library's sort rule, and the flop recount of the field kernel."""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sort_launch_rule_matches_the_library():
    src = open(os.path.join(ROOT, "paper_2111_13072_gb300", "csrc", "imrp_core.cu")).read()
    m = re.search(r"constexpr int64_t kBucketSortMaxN = (\d+);", src)
    assert m and int(m.group(1)) == bench.BUCKET_SORT_MAX_N
    m = re.search(r"constexpr int64_t kBsSingleN = (\d+);", src)
    assert m and int(m.group(1)) == bench.BUCKET_SORT_SINGLE_N
    assert bench.sort_launches(1) == 0
    assert bench.sort_launches(2) == 1
    assert bench.sort_launches(bench.BUCKET_SORT_SINGLE_N) == 1
    assert bench.sort_launches(bench.BUCKET_SORT_SINGLE_N + 1) == 4
    assert bench.sort_launches(bench.BUCKET_SORT_MAX_N) == 4
    assert bench.sort_launches(bench.BUCKET_SORT_MAX_N + 1) == 12
    assert bench.step_launches(2_000_000) == 11


def test_field_flop_recount():
    # far field: real column 10 per entry (+6), complex columns 16 per entry after
    # the first, 12 + 8 per column; near field 16 pairs; tail 50 + 2 L
    assert bench.field_flops_per_particle(16) == 8900
    assert bench.field_flops_per_particle(24) == 16052

"""Per-launch timeline of the profiler (raptor_profile_timeline): one record per profiled
launch scope, in launch order, consistent with the per-slot sums; a mixed render shows its
second stream's FP64 launches overlapping the first stream's phases.  Needs a GPU."""
import numpy as np
import pytest

from paper_1801_10452_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1801_10452_b300 import build

    build.build()
    import paper_1801_10452_b300 as R

    return R


def test_timeline_matches_slot_sums_and_shows_both_streams(R):
    import torch

    cam = dict(scenes.SMALL, nx=96, ny=96, precision=R.MIXED, flags=R.FLAG_INNER_DF64)
    ctx = R.Context(R.camera_desc(**cam))
    ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
    ctx.render([230e9])
    ctx.profile(True)
    ctx.render([230e9])
    torch.cuda.synchronize()
    tl = ctx.profile_timeline()
    sums = ctx.profile_read()
    ctx.profile(False)
    names = [t[0] for t in tl]
    # A1, A2, C, C-long; one FP64 launch on the second stream (its own slot) and eight passes;
    # two reductions
    assert names.count("mixed_fp32_in") == 2 and names.count("mixed_fp32_out") == 2
    assert names.count("reduce") == 2
    assert {t[1] for t in tl if t[0] == "mixed_fp64"} == {0}
    assert {t[1] for t in tl if t[0] == "mixed_fp64_long"} == {1}
    # the second stream's FP64 steps are counted apart, and are part of the FP64 steps
    st = ctx.stats_ex()
    assert 0 < st["fp64_steps_long"] < st["fp64_steps"]
    assert all(t[2] >= -0.05 and t[3] >= 0.0 for t in tl)
    for k, (ms, _) in sums.items():
        tot = sum(t[3] for t in tl if t[0] == k)
        assert abs(tot - ms) <= 1e-6 + 1e-9 * ms, k
    # stream order: on each lane the records start no earlier than the previous one ended
    for lane in (0, 1):
        rec = [t for t in tl if t[1] == lane]
        for a, b in zip(rec, rec[1:]):
            assert b[2] >= a[2] + a[3] - 0.01, (a, b)
    # phase C of B-long's leavers runs on the second stream after B-long, the other C on the
    # first; the join: the flux reduction starts after the second stream's last launch ended
    assert sorted(t[1] for t in tl if t[0] == "mixed_fp32_out") == [0, 1]
    c_long = [t for t in tl if t[0] == "mixed_fp32_out" and t[1] == 1][0]
    long_fp64_end = max(t[2] + t[3] for t in tl if t[0] == "mixed_fp64_long")
    assert c_long[2] >= long_fp64_end - 0.01
    long_end = max(t[2] + t[3] for t in tl if t[1] == 1)
    red = [t for t in tl if t[0] == "reduce"][0]
    assert red[2] >= long_end - 0.01
    # a second profile(True) clears the records
    ctx.profile(True)
    assert ctx.profile_timeline() == []
    ctx.profile(False)

"""Autotuner host logic (CPU) and one GPU tuning run."""
import pytest

from paper_1612_03804_gb300.tune import LIMIT, candidates


def test_candidates_respect_condition_bound_and_M():
    c = candidates(160, 0.05)
    assert c and max(c) * 0.05 * 10 <= LIMIT and max(c) <= 160
    assert candidates(4, 0.05) == [2, 3, 4]
    assert all(n * 0.1 * 10 <= LIMIT for n in candidates(100, 0.1))


@pytest.mark.gpu
def test_autotune_picks_an_accurate_candidate():
    import torch
    from paper_1612_03804_gb300 import build
    from paper_1612_03804_gb300.tune import TOL, autotune_nwrap
    build.build()
    torch.cuda.set_device(0)
    best, res = autotune_nwrap(12, 4.0, 0.05, -0.5, "3xtf32", batch=4, reps=1)
    assert best in [r[0] for r in res]
    assert dict((r[0], r[2]) for r in res)[best] <= TOL["3xtf32"]


@pytest.mark.gpu
def test_autotune_schedule_tries_both_tiles():
    import torch
    from paper_1612_03804_gb300 import build
    from paper_1612_03804_gb300.tune import TOL, autotune_schedule
    build.build()
    torch.cuda.set_device(0)
    nw, tile, res = autotune_schedule(12, 2.0, 0.05, -0.5, "3xtf32", batch=4, reps=1)
    assert {r[1] for r in res} == {64, 128}
    assert (nw, tile) in [(r[0], r[1]) for r in res]
    err = dict(((r[0], r[1]), r[3]) for r in res)
    assert err[(nw, tile)] <= TOL["3xtf32"]
    # every pair faster than the chosen one misses the bound
    ms = dict(((r[0], r[1]), r[2]) for r in res)
    assert all(err[k] > TOL["3xtf32"] for k in ms if ms[k] < ms[(nw, tile)])

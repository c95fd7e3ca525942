"""The autotuner on a small sample: every candidate of a grid that mixes the
direction rules and the BFS-side reduction must return the same r (and,
without reductions, the same words), and the best setting is one of the
grid's."""

import pytest

from paper_2207_05495_gb300 import gen

pytestmark = pytest.mark.gpu


def test_tune_small_grid():
    import torch
    assert torch.cuda.is_available()
    from paper_2207_05495_gb300 import autotune, build, sw
    build.build()
    sample = gen.batch_random(24, 40, 90, 2, 31)
    grid = {"set_cost": [512.0, 131072.0], "reduce": [0, 2], "dir_rule": [0, 1]}
    before = sw.sw_get_options()
    res = autotune.tune(sample, sw.workspace(1 << 30), grid=grid, repeats=1)
    assert len(res["trials"]) + res["pruned"] == 8 and res["complete"]
    assert res["best"] in [{k: t[k] for k in grid} for t in res["trials"]]
    after = sw.sw_get_options()  # the caller's options are restored
    assert (after.set_cost, after.reduce, after.dir_rule) == (before.set_cost, before.reduce, before.dir_rule)

"""The allocation-free entry point, sw_reset_threshold_static.

It is for callers that cannot allocate device memory when they call in (a
process whose allocator already holds the GPU, a plugin inside a program
that owns all device memory, a service that fixes its memory at start-up).
It must give the same r, word and level sizes as sw_reset_threshold, which
searches in a caller-provided workspace, and keep doing so on consecutive
calls that share its fixed device scratch.  This file is collected last.
"""

import numpy as np
import pytest

from paper_2207_05495_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2207_05495_gb300 import build, sw as swmod
    build.build()
    return swmod


def test_static_scratch_matches_workspace_path(sw):
    ws = sw.workspace(256 << 20)
    cases = [gen.random_automaton(40, 2, 0), gen.cerny(9), gen.random_automaton(60, 3, 5)]
    for d in cases:
        h = sw.load(d)
        want = sw.sw_reset_threshold(h, ws=ws)
        want_sizes = sw.sw_level_sizes(h)
        for _ in range(2):  # two calls in a row share the scratch
            got = sw.sw_reset_threshold_static(h)
            assert got == want  # integer results: exact
            assert sw.sw_level_sizes(h) == want_sizes


def test_static_scratch_rejects_too_large(sw):
    # a 576-state automaton with nine-word sets cannot fit 64 MiB of scratch
    d = gen.random_automaton(576, 2, 1)
    with pytest.raises(sw.SwError) as e:
        sw.sw_reset_threshold_static(sw.load(d))
    assert e.value.code == sw.SW_ENOMEM

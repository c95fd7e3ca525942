"""The allocation-free entry point, sw_reset_threshold_static.

It is for callers that cannot allocate device memory when they call in (a
process whose allocator already holds the GPU, a plugin inside a program
that owns all device memory, a service that fixes its memory at start-up).
It must give the same r, word and level sizes as sw_reset_threshold, which
searches in a caller-provided workspace, and as the CPU oracle, keep doing
so on consecutive calls that share its fixed device scratch, and leave the
device's free memory unchanged.  This file is collected last.
"""

import numpy as np
import pytest

import oracle
from paper_2207_05495_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2207_05495_gb300 import build, sw as swmod
    build.build()
    return swmod


CASES = [("n40", lambda: gen.random_automaton(40, 2, 0)), ("cerny9", lambda: gen.cerny(9)),
         ("n60k3", lambda: gen.random_automaton(60, 3, 5))]


def test_static_scratch_matches_workspace_path_and_oracle(sw):
    ws = sw.workspace(256 << 20)
    for name, make in CASES:
        d = make()
        h = sw.load(d)
        want = sw.sw_reset_threshold(h, ws=ws)
        want_sizes = sw.sw_level_sizes(h)
        ro, wo, _, _ = oracle.bidir(d)
        assert want == (ro, wo), name
        for _ in range(2):  # two calls in a row share the scratch
            got = sw.sw_reset_threshold_static(h)
            assert got == want, name  # integer results: exact
            assert sw.sw_level_sizes(h) == want_sizes, name


def test_static_scratch_allocates_no_device_memory(sw):
    import torch
    h = sw.load(gen.random_automaton(50, 2, 3))
    sw.sw_reset_threshold_static(h)  # loads the module; the scratch is then resident
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        sw.sw_reset_threshold_static(h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_exhausted_is_enomem(sw):
    # Every valid automaton passes the size check on entry; a 576-state
    # random automaton's search then outgrows the 64 MiB array (its levels
    # and tables), and the engine reports SW_ENOMEM once it has set back its
    # only instance.
    d = gen.random_automaton(576, 2, 1)
    with pytest.raises(sw.SwError) as e:
        sw.sw_reset_threshold_static(sw.load(d))
    assert e.value.code == sw.SW_ENOMEM
    # the scratch is still usable afterwards
    d = gen.cerny(7)
    assert sw.sw_reset_threshold_static(sw.load(d)) == oracle.bidir(d)[:2]

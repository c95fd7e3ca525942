"""Hard single instances: the random binary automata with n = 300 and
n = 400 states (seed 0; delta iid uniform, five and seven 64-bit words per
set), each searched alone with a large workspace.

Its reset threshold is out of the oracle's reach (about 10^7 sets per
direction and 10^14 candidate pairs at the meet), so the result is checked
by what holds at any size:
  - the word maps Q to one state and has length r;
  - r is at most the length of a reset word found by a plain beam search
    over images (the smallest sets of each level kept), an upper bound
    computed here on the CPU;
  - every forward level up to depth 20 and every backward level up to depth
    16 that the search computed has exactly the oracle's size;
  - two searches with different direction schedules (the paper's step-cost
    rule with the library's SetCost, and "expand the smaller side", a huge
    SetCost) return the same r and the same least word, and agree on the
    sizes of every level both computed.
"""

import numpy as np
import pytest

import oracle
from paper_2207_05495_gb300 import gen

pytestmark = pytest.mark.gpu

SEED = 0


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2207_05495_gb300 import build, sw as swmod
    build.build()
    return swmod


def beam_upper_bound(d, beam):
    """Length of the first reset word found by keeping, at every depth, the
    `beam` smallest distinct images (ties in generation order)."""
    k, n = d.shape
    cur = np.ones((1, n), bool)
    for depth in range(1, 4 * n):
        nxt = []
        for a in range(k):
            img = np.zeros_like(cur)
            rows, cols = np.nonzero(cur)
            img[rows, d[a][cols]] = True
            nxt.append(img)
        nxt = np.unique(np.concatenate(nxt), axis=0)
        card = nxt.sum(1)
        if card.min() == 1:
            return depth
        cur = nxt[np.argsort(card, kind="stable")[:beam]]
    raise AssertionError("beam search found no reset word")


def run(sw, ws, n, set_cost):
    old = sw.sw_get_options()
    o = sw.sw_get_options()
    o.set_cost = set_cost
    sw.sw_set_options(o)
    try:
        h = sw.load(gen.random_automaton(n, 2, SEED))
        r, w = sw.sw_reset_threshold(h, ws=ws)
        return r, w, sw.sw_level_sizes(h)
    finally:
        sw.sw_set_options(old)


@pytest.mark.parametrize("N", [300, 400])
def test_hard_single(sw, N):
    import torch
    d = gen.random_automaton(N, 2, SEED)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    ws = sw.workspace(min(200 << 30, int(free * 0.8)))
    r1, w1, (f1, b1) = run(sw, ws, N, sw.sw_get_options().set_cost)
    r2, w2, (f2, b2) = run(sw, ws, N, 1e9)
    del ws
    assert (r1, w1) == (r2, w2)
    assert len(w1) == r1
    st = np.arange(N)
    for a in w1:
        st = d[a][st]
    assert len(np.unique(st)) == 1
    assert r1 <= beam_upper_bound(d, 20000)
    for fa, fb in ((f1, f2), (b1, b2)):
        m = min(len(fa), len(fb))
        assert fa[:m] == fb[:m]
    fwd = max(f1, f2, key=len)
    bwd = max(b1, b2, key=len)
    df, db = min(20, len(fwd) - 1), min(16, len(bwd) - 1)
    assert fwd[: df + 1] == oracle.level_sizes(d, 0, df)
    assert bwd[: db + 1] == oracle.level_sizes(d, 1, db)
    assert len(f1) + len(b1) - 2 == r1 and len(f2) + len(b2) - 2 == r2

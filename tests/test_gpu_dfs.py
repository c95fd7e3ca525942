"""The memory-bounded inverse phase (sw_options.dfs_sets; Section 2.2):
once the bidirectional phase stops, chunks of the last inverse level are
expanded deeper and checked against the last forward level.

Against the CPU oracle, through the C-ABI: r is identical to the plain
bidirectional oracle's; the word resets and has length r; the levels of the
bidirectional phase equal the oracle's level sizes.  Whether the phase ran
is read from sw_last_dfs_stats and from the level sizes (their depths then
add up to less than r)."""

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


@pytest.fixture(scope="module")
def ws(sw):
    return sw.workspace(256 << 20)


def set_dfs(sw, sets):
    o = sw.sw_get_options()
    o.dfs_sets = sets
    sw.sw_set_options(o)


@pytest.fixture
def restore(sw):
    old = sw.sw_get_options()
    yield
    sw.sw_set_options(old)


def resets(delta, word):
    states = np.arange(delta.shape[1])
    for a in word:
        states = delta[a][states]
    return len(np.unique(states)) == 1


def check(sw, d, h, r, w):
    """Checks one result; returns True when the inverse phase produced it."""
    assert r == oracle.bidir(d)[0]
    assert len(w) == r and resets(d, w)
    fs, bs = sw.sw_level_sizes(h)
    assert fs == oracle.level_sizes(d, 0, len(fs) - 1)
    assert bs == oracle.level_sizes(d, 1, len(bs) - 1)
    return len(fs) + len(bs) - 2 < r


@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
def test_cerny(sw, ws, restore, n):
    set_dfs(sw, 12)
    d = gen.cerny(n)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    assert r == (n - 1) ** 2
    ran = check(sw, d, h, r, w)
    st = sw.sw_last_dfs_stats()
    assert ran == (st["dfs_instances"] == 1)
    if n >= 6:
        assert ran and st["dfs_chunks"] >= 1 and st["dfs_sets"] > 0


def _cases():
    rng = np.random.default_rng(2207)
    out = []
    for i in range(36):
        k = int(rng.choice([2, 2, 3, 4]))
        n = int(rng.integers(6, 70 if k == 2 else 40))
        budget = int(rng.choice([6, 20, 64, 300, 2000]))
        out.append((n, k, 3100 + i, budget))
    return out


@pytest.mark.parametrize("n,k,seed,budget", _cases())
def test_random_vs_oracle(sw, ws, restore, n, k, seed, budget):
    set_dfs(sw, budget)
    d = gen.random_automaton(n, k, seed)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    check(sw, d, h, r, w)


def test_small_budgets_run_the_phase(sw, ws, restore):
    # with a budget below the first levels' sizes, every instance with
    # r >= 4 goes through the inverse phase
    set_dfs(sw, 4)
    ran = 0
    for seed in range(20):
        d = gen.random_automaton(30, 2, 800 + seed)
        h = sw.load(d)
        r, w = sw.sw_reset_threshold(h, ws=ws)
        ran += check(sw, d, h, r, w)
    assert ran >= 15


def test_batch_with_budget(sw, ws, restore):
    # instances of one batch leave the bidirectional phase at different
    # iterations; each gets its inverse phase and the others go on
    set_dfs(sw, 150)
    ds = gen.batch_random(24, 20, 80, 2, 4400)
    hs = [sw.load(d) for d in ds]
    rb, wb = sw.sw_batch(hs, ws=ws)
    ran = sum(check(sw, d, hs[t], int(rb[t]), wb[t]) for t, d in enumerate(ds))
    assert ran >= 1
    assert sw.sw_last_dfs_stats()["dfs_instances"] == ran


def test_memory_exhausted(sw, restore):
    # workspaces too small for the bidirectional phase: without the inverse
    # phase the search ends with SW_ENOMEM; with it (dfs_sets = -1) it
    # finds the oracle's r, or ends with SW_ENOMEM itself when not even one
    # root's expansion fits
    seen = 0
    base = int(sw.lib().sw_workspace_min_bytes(64, 2, 1))
    for seed in range(10):
        d = gen.random_automaton(64, 2, 5100 + seed)
        h = sw.load(d)
        for mult in (1, 2, 4):
            small = sw.workspace(base * mult)
            set_dfs(sw, 0)
            try:
                sw.sw_reset_threshold(h, ws=small)
                continue  # it fitted
            except sw.SwError as e:
                assert e.code == sw.SW_ENOMEM
            set_dfs(sw, -1)
            try:
                r, w = sw.sw_reset_threshold(h, ws=small)
            except sw.SwError as e:
                assert e.code == sw.SW_ENOMEM
                continue
            assert check(sw, d, h, r, w)
            seen += 1
    assert seen >= 1


@pytest.mark.parametrize("reduce_mode", [1, 2, 3], ids=["both", "bfs", "ibfs"])
def test_after_reduced_phase(sw, ws, restore, reduce_mode):
    # the inverse phase after a reduced bidirectional phase: F_i and B_j
    # hold a subset (superset) of every set first reached at their depths,
    # so r is still the oracle's; the word resets and has length r
    o = sw.sw_get_options()
    o.reduce = reduce_mode
    o.dfs_sets = 40
    sw.sw_set_options(o)
    ran = 0
    for seed in range(8):
        d = gen.random_automaton(36, 2, 6200 + seed)
        h = sw.load(d)
        r, w = sw.sw_reset_threshold(h, ws=ws)
        assert r == oracle.bidir(d)[0]
        assert len(w) == r and resets(d, w)
        fs, bs = sw.sw_level_sizes(h)
        ran += len(fs) + len(bs) - 2 < r
    assert ran >= 1

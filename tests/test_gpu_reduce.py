"""GPU search with the inclusion reductions of Alg. 1 (sw_options.reduce = 1:
both sides; 2: the BFS side; 3: the IBFS side) against the CPU oracle's
restatement (oracle.bidir_reduced with the same sides), element by
element, through the C-ABI.

r and every computed reduced level size must be identical.  The word of
the reduced search depends on the forward depth at which the two searches
met (the level sizes give it), so the oracle is run with that split and
its word must be identical too; it is also checked to be a reset word of
length r.  The r of the reduced search must equal the plain search's."""

import functools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2207_05495_gb300 import gen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2207_05495_gb300 import build, sw as swmod
    build.build()
    return swmod


@pytest.fixture(scope="module")
def ws(sw):
    return sw.workspace(512 << 20)


SIDES = {1: 3, 2: 1, 3: 2}  # sw_options.reduce -> the oracle's side mask


@pytest.fixture(params=[1, 2, 3], ids=["both", "bfs", "ibfs"])
def reduced(sw, request):
    old = sw.sw_get_options()
    o = sw.sw_get_options()
    o.reduce = request.param
    sw.sw_set_options(o)
    yield SIDES[request.param]
    sw.sw_set_options(old)


def resets(delta, word):
    states = np.arange(delta.shape[1])
    for a in word:
        states = delta[a][states]
    return len(np.unique(states)) == 1


def check(sw, d, h, r, w, dirs):
    fs, bs = sw.sw_level_sizes(h)
    i = len(fs) - 1
    ro, wo, fo, bo = oracle.bidir_reduced(d, fwd_depth=i, dirs=dirs)
    assert r == ro and len(fs) + len(bs) - 2 == r
    assert w == wo and resets(d, w)
    assert fs == fo and bs == bo


def test_hand_examples(sw, ws, reduced):
    for ex in json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["examples"]:
        d = np.array(ex["delta"], dtype=np.int32)
        h = sw.load(d)
        r, w = sw.sw_reset_threshold(h, ws=ws)
        assert r == ex["r"], ex["name"]
        check(sw, d, h, r, w, reduced)


@pytest.mark.parametrize("n", list(range(1, 21)))
def test_cerny(sw, ws, reduced, n):
    d = gen.cerny(n)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    assert r == (n - 1) ** 2
    check(sw, d, h, r, w, reduced)


def _random_cases():
    cases = []
    rng = np.random.default_rng(4242)
    for i in range(40):
        n = int(rng.integers(2, 64))
        k = int(rng.choice([1, 2, 2, 3, 4]))
        cases.append((n, k, 11000 + i))
    return cases


@pytest.mark.parametrize("n,k,seed", _random_cases())
def test_random_vs_oracle(sw, ws, reduced, n, k, seed):
    d = gen.random_automaton(n, k, seed)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    assert r == oracle.bidir(d)[0]
    check(sw, d, h, r, w, reduced)


@pytest.mark.parametrize("n,m,k,seed", [(250, 40, 3, 4), (330, 48, 2, 7), (450, 50, 2, 5), (576, 44, 2, 3)])
def test_wide_sets_vs_oracle(sw, ws, reduced, n, m, k, seed):
    # sets spread over four to nine words (gen.core_automaton)
    d = gen.core_automaton(n, m, k, seed)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    check(sw, d, h, r, w, reduced)


def test_max_letters(sw, ws, reduced):
    for n, seed in ((8, 1), (12, 2)):
        d = gen.random_automaton(n, sw.SW_MAX_LETTERS, seed)
        h = sw.load(d)
        r, w = sw.sw_reset_threshold(h, ws=ws)
        check(sw, d, h, r, w, reduced)


def test_ragged_batch(sw, ws, reduced):
    # one batch mixing n = 1 .. 100 and k = 1 .. 4; every instance against
    # the oracle with its own split
    rng = np.random.default_rng(6)
    ds = [gen.random_automaton(1, 3, 1), gen.random_automaton(4, 1, 2)]
    while len(ds) < 32:
        k = int(rng.integers(2, 5))
        n = int(rng.integers(2, 100 if k == 2 else 50))
        ds.append(gen.random_automaton(n, k, 1900 + len(ds)))
    hs = [sw.load(d) for d in ds]
    rb, wb = sw.sw_batch(hs, ws=ws)
    for i, d in enumerate(ds):
        check(sw, d, hs[i], int(rb[i]), wb[i], reduced)


@functools.lru_cache(maxsize=None)
def _c3_golden():
    with open(os.path.join(GOLDEN, "c3_sample.json")) as fh:
        return json.load(fh)


def test_c3_sample_reduced_r_and_sizes(sw, reduced):
    # instances of the 4096-automaton workload: r equals the stored oracle
    # r (written by the plain bidirectional oracle), and the reduced level
    # sizes of the smaller ones equal the oracle's reduced sizes
    g = _c3_golden()
    items = g["instances"][:24]
    ds = [gen.random_automaton_ranged(64, 192, 2, it["seed"]) for it in items]
    hs = [sw.load(d) for d in ds]
    ws = sw.workspace(8 << 30)
    rb, wb = sw.sw_batch(hs, ws=ws, word_cap=1024)
    for i, it in enumerate(items):
        assert int(rb[i]) == it["r"], it["seed"]
        assert len(wb[i]) == it["r"] and resets(ds[i], wb[i])
        if ds[i].shape[1] <= 90:
            fs, bs = sw.sw_level_sizes(hs[i])
            side = lambda dr, depth: (oracle.reduced_level_sizes if reduced & (1 << dr)  # noqa: E731
                                      else oracle.level_sizes)(ds[i], dr, depth)
            assert fs == side(0, len(fs) - 1)
            assert bs == side(1, len(bs) - 1)


def test_reduced_equals_plain_r_in_waves(sw, reduced):
    # a workspace too small for all instances at once: set-backs and waves
    # in reduced mode give the same r as a roomy run
    ds = gen.batch_random(48, 64, 128, 2, 700)
    hs = [sw.load(d) for d in ds]
    r_big, _ = sw.sw_batch(hs, ws=sw.workspace(1 << 30))
    for mib in (16, 24, 32, 48, 64, 96):
        r_small, w_small = sw.sw_batch(hs, ws=sw.workspace(mib << 20), raise_on_error=False)
        ok = r_small >= 0
        assert (r_small[ok] == r_big[ok]).all()
        assert all(resets(ds[i], w_small[i]) for i in np.nonzero(ok)[0])
        if ok.all():
            break

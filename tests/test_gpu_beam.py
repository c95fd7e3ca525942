"""The GPU beam upper bound (sw_beam, Section 2.1.3) against the CPU
oracle's restatement (oracle.beam): R and the word must be identical (the
cut and every tie-break are fixed: largest sets first, then candidate
order), R >= r, and the word must reset Q.  Calls go through the C-ABI."""

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
    return sw.workspace(1 << 30)


def resets(delta, word):
    states = np.arange(delta.shape[1])
    for a in word:
        states = delta[a][states]
    return len(np.unique(states)) == 1


def _cases():
    rng = np.random.default_rng(808)
    out = []
    for i in range(30):
        n = int(rng.integers(2, 120))
        k = int(rng.choice([2, 2, 3]))
        B = int(rng.choice([2, 8, 64, 1000]))
        out.append((n, k, B, 3000 + i))
    return out


@pytest.mark.parametrize("n,k,B,seed", _cases())
def test_beam_vs_oracle(sw, ws, n, k, B, seed):
    d = gen.random_automaton(n, k, seed)
    try:
        want = oracle.beam(d, B, max_depth=4 * n)
    except oracle.OracleError as e:  # a small beam that cycles: both must say so
        with pytest.raises(sw.SwError) as g:
            sw.sw_beam(d, B, ws=ws, max_depth=4 * n)
        assert g.value.code == sw.SW_ENOTFOUND and e.code == -6
        return
    R, w = sw.sw_beam(d, B, ws=ws, max_depth=4 * n)
    assert (R, w) == want[:2]
    assert resets(d, w) and R >= oracle.bidir(d)[0] if n <= 60 else resets(d, w)


@pytest.mark.parametrize("n", [2, 5, 9, 16])
def test_beam_cerny_without_cut(sw, ws, n):
    d = gen.cerny(n)
    R, w = sw.sw_beam(d, 1 << 40, ws=ws)
    assert R == (n - 1) ** 2 and resets(d, w)
    assert (R, w) == oracle.beam(d, 1 << 40)[:2]


@pytest.mark.parametrize("n,B", [(700, 200), (1500, 64), (3000, 32)])
def test_beam_large_automata(sw, ws, n, B):
    # sets of 11 to 47 words: beyond the exact search's 576 states
    d = gen.random_automaton(n, 2, 1)
    R, w = sw.sw_beam(d, B, ws=ws, max_depth=8 * n)
    assert (R, w) == oracle.beam(d, B, max_depth=8 * n)[:2]
    assert resets(d, w)


def test_beam_is_upper_bound_on_hard_instances(sw, ws):
    # the exact r of these (n = 300: 50, n = 400: 51) comes from the GPU
    # search's tests; the beam of size n log n must not undercut it
    for n, r in ((300, 50), (400, 51)):
        d = gen.random_automaton(n, 2, 0)
        B = int(n * np.ceil(np.log2(n)))
        R, w = sw.sw_beam(d, B, ws=ws)
        assert R >= r and resets(d, w)

"""The seeded input generator: stream values, determinism, the recipe."""

import numpy as np

from paper_2207_05495_gb300 import gen


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    assert [int(x) for x in gen.splitmix64_block(0, 0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_blocks_concatenate():
    whole = gen.splitmix64_block(7, 0, 10)
    parts = np.concatenate([gen.splitmix64_block(7, 0, 4), gen.splitmix64_block(7, 4, 6)])
    assert (whole == parts).all()


def test_below_is_exact_multiply_shift():
    x = gen.splitmix64_block(3, 0, 1000)
    for m in (1, 2, 3, 40, 192, 576):
        ref = [(int(v) * m) >> 64 for v in x]
        assert gen.below(x, m).tolist() == ref


def test_random_automaton_deterministic_and_synchronizing():
    a = gen.random_automaton(40, 2, 0)
    b = gen.random_automaton(40, 2, 0)
    assert (a == b).all() and a.shape == (2, 40) and a.dtype == np.int32
    assert gen.is_synchronizing(a)
    assert a.min() >= 0 and a.max() < 40


def test_ranged_sizes():
    ns = [gen.random_automaton_ranged(64, 192, 2, s).shape[1] for s in range(64)]
    assert min(ns) >= 64 and max(ns) <= 192 and len(set(ns)) > 20


def test_cerny_shape():
    c = gen.cerny(5)
    assert c.tolist() == [[1, 2, 3, 4, 0], [1, 1, 2, 3, 4]]


def test_core_automaton_lands_in_a_scattered_core():
    d = gen.core_automaton(300, 40, 2, 1)
    assert (d == gen.core_automaton(300, 40, 2, 1)).all() and d.shape == (2, 300)
    core = np.unique(d)
    assert len(core) <= 40 and core.min() >= 0 and core.max() < 300
    # the core is spread over all five 64-bit words of a 300-state set
    assert len(set((core // 64).tolist())) == 5
    assert gen.is_synchronizing(d)

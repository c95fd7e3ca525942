"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these checks reuses the oracle's own code: hand derivations
(tests/golden/hand_examples.json), the closed form for Cerny automata
(Section 1.1), the definition of a reset word (Section 1) applied directly
with numpy, brute-force enumeration of words in plain Python, exhaustive
enumeration of all small binary automata, and bounds (Frankl-Pin, Section
1.1; sink automata, Section 3.1.1).
"""

import itertools
import json
import os

import numpy as np
import pytest

import oracle
from paper_2207_05495_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def resets(delta, word):
    """|delta(Q, w)| == 1, straight from the definition (Section 1)."""
    delta = np.asarray(delta)
    states = np.arange(delta.shape[1])
    for a in word:
        states = delta[a][states]
    return len(np.unique(states)) == 1


def brute_levels(delta, direction, depth):
    """Deduplicated level sizes by enumerating every word (plain Python).

    Forward: D_i = {delta(Q, w) : |w| = i}; level i = D_i minus every
    D_i' with i' < i.  Backward: E_j = nonempty {delta^{-1}({q}, y) : |y| = j};
    level j = E_j minus every earlier E_j'."""
    delta = [list(map(int, row)) for row in np.asarray(delta)]
    k, n = len(delta), len(delta[0])
    seen, sizes = set(), []
    for d in range(depth + 1):
        cur = set()
        for w in itertools.product(range(k), repeat=d):
            if direction == 0:
                s = set(range(n))
                for a in w:
                    s = {delta[a][q] for q in s}
                cur.add(frozenset(s))
            else:
                for q in range(n):
                    s = {q}
                    for a in reversed(w):  # delta^{-1}({q}, w) = pre(...pre({q}, w_last)...)
                        s = {p for p in range(n) if delta[a][p] in s}
                    if s:
                        cur.add(frozenset(s))
        new = cur - seen
        sizes.append(len(new))
        seen |= cur
    return sizes


def cerny_word(n):
    """b (a^{n-1} b)^{n-2}: each a^{n-1} b removes one state of {1..m}."""
    return [] if n == 1 else [1] + ([0] * (n - 1) + [1]) * (n - 2)


# ---------------------------------------------------------------- hand examples

with open(os.path.join(GOLDEN, "hand_examples.json")) as fh:
    HAND = json.load(fh)["examples"]


@pytest.mark.parametrize("ex", HAND, ids=[e["name"] for e in HAND])
def test_hand_examples(ex):
    d = np.array(ex["delta"], dtype=np.int32)
    r, w, fs = oracle.forward(d)
    assert r == ex["r"] and w == ex["word"]
    assert fs == ex["fwd_sizes"]
    assert oracle.level_sizes(d, 1, len(ex["bwd_sizes"]) - 1) == ex["bwd_sizes"]
    rb, wb, fsb, bsb = oracle.bidir(d)
    assert (rb, wb) == (ex["r"], ex["word"])
    assert fsb == ex["fwd_sizes"][: len(fsb)]
    assert bsb == ex["bwd_sizes"][: len(bsb)]
    assert oracle.brute(d, 8) == (ex["r"], ex["word"])


# ---------------------------------------------------------------- Cerny closed form

@pytest.mark.parametrize("n", range(1, 17))
def test_cerny_forward_closed_form(n):
    d = gen.cerny(n)
    r, w, _ = oracle.forward(d)
    assert r == (n - 1) ** 2
    assert w == cerny_word(n)
    assert resets(d, w)


@pytest.mark.parametrize("n", range(1, 6))
def test_cerny_brute_unique_word(n):
    # brute force returns the least word; the closed-form word is the least
    d = gen.cerny(n)
    assert oracle.brute(d, (n - 1) ** 2) == ((n - 1) ** 2, cerny_word(n))


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12, 16, 20])
def test_cerny_bidirectional(n):
    d = gen.cerny(n)
    r, w, _, _ = oracle.bidir(d)
    assert r == (n - 1) ** 2 and w == cerny_word(n)


# ---------------------------------------------------------------- brute force

def _small_random(count, n_range, k_range, seed0):
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        out.append(gen.random_automaton(n, k, seed0 * 1000 + i))
    return out


@pytest.mark.parametrize("d", _small_random(40, (2, 7), (1, 3), 11))
def test_forward_equals_brute(d):
    rb, wb = oracle.brute(d, 16)
    r, w, _ = oracle.forward(d)
    assert (r, w) == (rb, wb)
    assert resets(d, w)


@pytest.mark.parametrize("d", _small_random(12, (2, 5), (1, 3), 23))
def test_level_sizes_equal_word_enumeration(d):
    depth = 5
    for direction in (0, 1):
        assert oracle.level_sizes(d, direction, depth) == brute_levels(d, direction, depth)


def test_all_binary_automata_n2_n3():
    """Every binary automaton on 2 and 3 states: the oracle's forward BFS,
    brute force and pair check agree with the input filter, and on 2
    states exactly the 12 automata with a constant letter synchronize, each
    with r = 1."""
    for n in (2, 3):
        count = 0
        for flat in itertools.product(range(n), repeat=2 * n):
            d = np.array(flat, dtype=np.int32).reshape(2, n)
            sync = gen.is_synchronizing(d)
            assert oracle.is_synchronizing(d) == sync
            if not sync:
                with pytest.raises(oracle.OracleError):
                    oracle.forward(d)
                continue
            count += 1
            r, w, _ = oracle.forward(d)
            assert oracle.brute(d, (n - 1) ** 2) == (r, w)
            if n == 2:
                assert r == 1
        if n == 2:
            assert count == 12


def test_all_binary_automata_n4_bound():
    """All 4^8 binary automata on 4 states: forward BFS and brute force
    agree, and the largest reset threshold is 9 = (n-1)^2 (the Cerny bound
    holds for 4 states, reached by C_4)."""
    best = 0
    for flat in itertools.product(range(4), repeat=8):
        d = np.array(flat, dtype=np.int32).reshape(2, 4)
        if not oracle.is_synchronizing(d):
            continue
        r, w, _ = oracle.forward(d)
        if r >= 6:  # brute force where it is cheap to compare the words too
            assert oracle.brute(d, 9) == (r, w)
        best = max(best, r)
    assert best == 9


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("d", _small_random(25, (8, 36), (2, 3), 37))
def test_bidirectional_equals_forward(d):
    r, w, fs = oracle.forward(d)
    rb, wb, fsb, bsb = oracle.bidir(d)
    assert (rb, wb) == (r, w)
    assert fsb == fs[: len(fsb)]
    assert bsb == oracle.level_sizes(d, 1, len(bsb) - 1)
    assert len(fsb) - 1 + len(bsb) - 1 == r
    assert resets(d, wb)
    n = d.shape[1]
    assert r <= (n ** 3 - n) // 6  # Frankl-Pin (Section 1.1)


@pytest.mark.parametrize("seed", range(10))
def test_sink_automata_bound(seed):
    n = 6 + seed
    d = gen.random_automaton(n, 2, 500 + seed, sink=True)
    r, w, _ = oracle.forward(d)
    assert r <= n * (n - 1) // 2  # Section 3.1.1: sink automata
    assert resets(d, w)
    s = np.arange(n)
    for a in w:
        s = d[a][s]
    assert set(s.tolist()) == {0}  # a reset word of a sink automaton ends in the sink


def test_one_state():
    d = np.zeros((2, 1), dtype=np.int32)
    assert oracle.forward(d) == (0, [], [1])
    assert oracle.bidir(d)[:2] == (0, [])
    assert oracle.brute(d, 4) == (0, [])


def test_rejects_bad_input():
    with pytest.raises(oracle.OracleError):
        oracle.forward(np.array([[0, 5]], dtype=np.int32))
    assert not oracle.is_synchronizing(np.array([[1, 0], [0, 1]], dtype=np.int32))


# ---------------------------------------------------------------- inclusion reductions (Alg. 1)

def reachable_by_depth(delta, direction, depth):
    """R[i] = the sets reachable at depth exactly i, from the definition:
    forward {delta(Q, w) : |w| = i}; backward the nonempty
    {delta^{-1}({q}, y) : |y| = i}.  Plain Python word enumeration."""
    delta = [list(map(int, row)) for row in np.asarray(delta)]
    k, n = len(delta), len(delta[0])
    out = []
    for d in range(depth + 1):
        cur = set()
        for w in itertools.product(range(k), repeat=d):
            if direction == 0:
                s = set(range(n))
                for a in w:
                    s = {delta[a][q] for q in s}
                cur.add(frozenset(s))
            else:
                for q in range(n):
                    s = {q}
                    for a in reversed(w):
                        s = {p for p in range(n) if delta[a][p] in s}
                    if s:
                        cur.add(frozenset(s))
        out.append(cur)
    return out


def reduced_levels_by_definition(delta, direction, depth):
    """The reduced level i, characterised without the search's recursion:
    forward, the sets S reachable at depth i with no set reachable at depth
    i that is a proper subset of S and no set reachable at a smaller depth
    that is a subset of S; backward, the same with supersets.  (A reachable
    set that the reduced search drops always has a kept subset -- superset
    backward -- at the same or a smaller depth, because images and
    preimages are monotone under inclusion; so the kept sets are exactly
    these.)"""
    R = reachable_by_depth(delta, direction, depth)
    below = lambda a, b: a <= b if direction == 0 else a >= b  # noqa: E731  a "beats" b
    levels = []
    earlier = set()
    for i in range(depth + 1):
        keep = set()
        for S in R[i]:
            if any(below(T, S) for T in earlier):
                continue
            if any(T != S and below(T, S) for T in R[i]):
                continue
            keep.add(S)
        levels.append(keep)
        earlier |= R[i]
    return levels


@pytest.mark.parametrize("d", _small_random(14, (2, 6), (1, 3), 61))
def test_reduced_level_sizes_equal_definition(d):
    depth = 5
    for direction in (0, 1):
        want = [len(L) for L in reduced_levels_by_definition(d, direction, depth)]
        assert oracle.reduced_level_sizes(d, direction, depth) == want


def test_reduced_level_sizes_all_binary_n3():
    for flat in itertools.product(range(3), repeat=6):
        d = np.array(flat, dtype=np.int32).reshape(2, 3)
        for direction in (0, 1):
            want = [len(L) for L in reduced_levels_by_definition(d, direction, 4)]
            assert oracle.reduced_level_sizes(d, direction, 4) == want


def plain_levels_by_definition(delta, direction, depth):
    """Level i without reductions: the sets reachable at depth i and at no
    smaller depth (duplicates and the equality history removed)."""
    R = reachable_by_depth(delta, direction, depth)
    out, earlier = [], set()
    for i in range(depth + 1):
        out.append(R[i] - earlier)
        earlier |= R[i]
    return out


def side_levels(delta, direction, depth, reduced):
    return (reduced_levels_by_definition if reduced else plain_levels_by_definition)(delta, direction, depth)


def reduced_word_by_definition(delta, r, i, dirs=3):
    """The reduced search's word for the split (i, r - i), by enumeration:
    x = the lexicographically least word of length i all of whose prefixes
    (x itself included) reach a kept set of their depth and whose set lies
    inside some kept backward set of depth r - i; then the least y of
    length r - i with |delta(delta(Q, x), y)| = 1.  dirs: which sides are
    reduced (bit 0 BFS, bit 1 IBFS); a plain side keeps the sets first
    reached at each depth."""
    dl = [list(map(int, row)) for row in np.asarray(delta)]
    k, n = len(dl), len(dl[0])
    j = r - i
    F = side_levels(delta, 0, i, dirs & 1)
    B = side_levels(delta, 1, j, dirs & 2)[j]
    for x in itertools.product(range(k), repeat=i):
        s = frozenset(range(n))
        ok = s in F[0]
        for t, a in enumerate(x):
            s = frozenset(dl[a][q] for q in s)
            ok = ok and s in F[t + 1]
        if ok and any(s <= Y for Y in B):
            for y in itertools.product(range(k), repeat=j):
                u = set(s)
                for a in y:
                    u = {dl[a][q] for q in u}
                if len(u) == 1:
                    return list(x) + list(y)
    raise AssertionError("no reduced word")


@pytest.mark.parametrize("d", _small_random(16, (3, 7), (2, 3), 71))
def test_reduced_search_r_word_and_sizes(d):
    rb, wb = oracle.brute(d, 16)
    r, w, fs, bs = oracle.bidir_reduced(d)
    assert r == rb and len(w) == r and resets(d, w)
    assert fs == [len(L) for L in reduced_levels_by_definition(d, 0, len(fs) - 1)]
    assert bs == [len(L) for L in reduced_levels_by_definition(d, 1, len(bs) - 1)]
    assert len(fs) + len(bs) - 2 == r
    assert w == reduced_word_by_definition(d, r, len(fs) - 1)
    for i in range(r + 1):  # every split: same r, the word of that split
        ri, wi, fi, bi = oracle.bidir_reduced(d, fwd_depth=i)
        assert ri == r and len(fi) - 1 == i and len(bi) - 1 == r - i
        assert wi == reduced_word_by_definition(d, r, i)
    # a split with no forward step gives the least reset word of all
    assert oracle.bidir_reduced(d, fwd_depth=0)[1] == wb


@pytest.mark.parametrize("dirs", [1, 2])
@pytest.mark.parametrize("d", _small_random(10, (3, 7), (2, 3), 77))
def test_one_side_reduced_search(d, dirs):
    # only one side reduced: that side's levels follow the reduced
    # characterisation, the other side's the plain one; r and the word of
    # every split as the enumeration says
    rb, wb = oracle.brute(d, 16)
    r, w, fs, bs = oracle.bidir_reduced(d, dirs=dirs)
    assert r == rb and resets(d, w)
    assert fs == [len(L) for L in side_levels(d, 0, len(fs) - 1, dirs & 1)]
    assert bs == [len(L) for L in side_levels(d, 1, len(bs) - 1, dirs & 2)]
    for i in range(r + 1):
        ri, wi, fi, bi = oracle.bidir_reduced(d, fwd_depth=i, dirs=dirs)
        assert ri == r and wi == reduced_word_by_definition(d, r, i, dirs)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12])
def test_reduced_cerny_closed_form(n):
    d = gen.cerny(n)
    r, w, _, _ = oracle.bidir_reduced(d)
    assert r == (n - 1) ** 2 and resets(d, w)
    assert oracle.bidir_reduced(d, fwd_depth=0)[1] == cerny_word(n)


@pytest.mark.parametrize("d", _small_random(10, (20, 40), (2, 3), 83))
def test_reduced_r_equals_unreduced(d):
    r, _, _, _ = oracle.bidir(d)
    rr, wr, fs, bs = oracle.bidir_reduced(d)
    assert rr == r and resets(d, wr)
    full_f = oracle.level_sizes(d, 0, len(fs) - 1)
    full_b = oracle.level_sizes(d, 1, len(bs) - 1)
    assert all(a <= b for a, b in zip(fs, full_f)) and all(a <= b for a, b in zip(bs, full_b))


# ---------------------------------------------------------------- beam upper bound (Section 2.1.3)

def beam_by_definition(delta, B, max_depth):
    """The cut-off inverse BFS in plain Python: level 0 = the singletons in
    order; each level = the distinct nonempty preimages of the previous
    level's sets in candidate order (parent position, then letter), of
    which the B largest are kept (ties: earlier candidate first), in
    candidate order; returns (R, sizes) for the first level holding Q."""
    dl = [list(map(int, row)) for row in np.asarray(delta)]
    k, n = len(dl), len(dl[0])
    cur = [frozenset([q]) for q in range(n)]
    sizes = [len(cur)]
    if n == 1:
        return 0, sizes
    for depth in range(1, max_depth + 1):
        seen, cands = set(), []
        for S in cur:
            for a in range(k):
                T = frozenset(p for p in range(n) if dl[a][p] in S)
                if T and T not in seen:
                    seen.add(T)
                    cands.append(T)
        order = sorted(range(len(cands)), key=lambda i: (-len(cands[i]), i))[:B]
        cur = [cands[i] for i in sorted(order)]
        sizes.append(len(cur))
        if any(len(S) == n for S in cur):
            return depth, sizes
    return None, sizes


@pytest.mark.parametrize("d", _small_random(20, (3, 9), (2, 3), 91))
def test_beam_equals_definition_and_bounds_r(d):
    r = oracle.brute(d, 20)[0]
    for B in (2, 3, 5, 1 << 30):
        want_R, want_sizes = beam_by_definition(d, B, 40)
        if want_R is None:
            with pytest.raises(oracle.OracleError):
                oracle.beam(d, B, max_depth=40)
            continue
        R, w, sizes = oracle.beam(d, B, max_depth=40)
        assert (R, sizes) == (want_R, want_sizes)
        assert len(w) == R and resets(d, w) and R >= r
        if B == 1 << 30:  # no cut: the inverse BFS reaches Q first at depth r
            assert R == r


@pytest.mark.parametrize("n", [2, 4, 7, 10])
def test_beam_cerny(n):
    d = gen.cerny(n)
    R, w, _ = oracle.beam(d, 1 << 30)
    assert R == (n - 1) ** 2 and resets(d, w)
    R1, w1, sizes = oracle.beam(d, 1)  # a beam of one still finds a word here
    assert R1 >= (n - 1) ** 2 and resets(d, w1) and max(sizes[1:] or [1]) == 1


# ---------------------------------------------------------------- O5: the inverse DFS phase


def _splits(r, span):
    """Every split (i, j) with i + j <= r and at most `span` inverse steps left."""
    return [(i, j) for i in range(r + 1) for j in range(r + 1 - i) if r - i - j <= span]


def test_inverse_dfs_from_any_split_gives_r():
    # Section 2.2: from the last levels F_i, B_j of any split below the
    # meet, the inverse phase finds r exactly (O1's r; a phase that used
    # images, tested Y inside X, or counted D off by one fails here)
    rng = np.random.default_rng(55)
    for t in range(30):
        k = int(rng.choice([2, 3]))
        n = int(rng.integers(3, 10))
        d = gen.random_automaton(n, k, 900 + t)
        r = oracle.forward(d)[0]
        for i, j in _splits(r, 8 if k == 2 else 5):
            assert oracle.inverse_dfs_r(d, i, j, max_depth=r) == r, (n, k, t, i, j)


def test_inverse_dfs_cerny():
    # r = (n - 1)^2 (Section 1.1) from splits up to ten inverse steps short
    for n in range(3, 7):
        d = gen.cerny(n)
        r = (n - 1) ** 2
        for i, j in _splits(r, 10):
            assert oracle.inverse_dfs_r(d, i, j, max_depth=r) == r, (n, i, j)


def test_inverse_dfs_every_binary_three_state_automaton():
    import itertools
    seen = 0
    for a in itertools.product(range(3), repeat=3):
        for b in itertools.product(range(3), repeat=3):
            d = np.array([a, b], dtype=np.int32)
            if not oracle.is_synchronizing(d):
                continue
            r = oracle.forward(d)[0]
            for i, j in _splits(r, r):
                assert oracle.inverse_dfs_r(d, i, j, max_depth=r) == r, (a, b, i, j)
            seen += 1
    assert seen > 100


def test_inverse_dfs_not_found_below_the_needed_depth():
    # the phase is exact: capped one step short of r it reports no meet
    d = gen.cerny(5)
    assert oracle.inverse_dfs_r(d, 3, 4, max_depth=16 - 7) == 16
    with pytest.raises(oracle.OracleError):
        oracle.inverse_dfs_r(d, 3, 4, max_depth=16 - 7 - 1)


def test_inverse_dfs_after_reduced_levels_gives_r():
    # the phase may start from reduced levels (Alg. 1's inclusion reductions
    # on either side): each kept level holds a subset (BFS) or superset
    # (IBFS) of every set first reached at its depth, so from any split
    # below the meet it still finds r
    rng = np.random.default_rng(77)
    for t in range(20):
        k = int(rng.choice([2, 3]))
        n = int(rng.integers(3, 9))
        d = gen.random_automaton(n, k, 1300 + t)
        r = oracle.forward(d)[0]
        for dirs in (1, 2, 3):
            for i, j in _splits(r, 7 if k == 2 else 4):
                assert oracle.inverse_dfs_r(d, i, j, dirs=dirs, max_depth=r) == r, (n, k, t, dirs, i, j)


# ---------------------------------------------------------------- O6: MarkSupersets (Alg. 2)


def _random_sets(rng, n, m, density):
    """m random subsets of {0..n-1} as uint64 [m][W] bitsets."""
    W = (n + 63) // 64
    bits = rng.random((m, n)) < density
    out = np.zeros((m, W), np.uint64)
    for q in range(n):
        out[:, q // 64] |= bits[:, q].astype(np.uint64) << np.uint64(q % 64)
    return out


def _lex_sorted_unique(sets, n):
    # lexicographic order of characteristic vectors from state 0 upwards,
    # absent before present (the order Alg. 2 requires of A)
    def key(row):
        return tuple(int((int(row[q // 64]) >> (q % 64)) & 1) for q in range(n))
    rows = {key(r): r for r in sets}
    return np.array([rows[k] for k in sorted(rows)], dtype=np.uint64).reshape(-1, sets.shape[1])


def _brute_marks(A, B, proper):
    marks = np.zeros(len(B), bool)
    for b, Y in enumerate(B):
        for X in A:
            if not np.any(X & ~Y) and not (proper and np.array_equal(X, Y)):
                marks[b] = True
                break
    return marks


@pytest.mark.parametrize("n", [1, 5, 13, 64, 70, 130])
def test_mark_supersets_equals_brute_force(n):
    rng = np.random.default_rng(n)
    for trial in range(12):
        dens_a, dens_b = rng.uniform(0.05, 0.6), rng.uniform(0.3, 0.95)
        A = _lex_sorted_unique(_random_sets(rng, n, int(rng.integers(0, 80)), dens_a), n)
        B = _random_sets(rng, n, int(rng.integers(0, 120)), dens_b)
        if len(A) and len(B):
            B[: len(B) // 4] = A[rng.integers(0, len(A), len(B) // 4)]  # some equal pairs
        for proper in (False, True):
            want = _brute_marks(A, B, proper)
            for mb in (1, 2, 8, 1000):  # the brute-force cut-off changes nothing
                got = oracle.mark_supersets(n, A, B, proper=proper, min_brute=mb)
                assert (got == want).all(), (n, trial, proper, mb)


def test_mark_subsets_by_complements():
    # MarkSubsets (the IBFS side) is MarkSupersets on the complements
    rng = np.random.default_rng(9)
    n = 40
    full = np.array([(1 << n) - 1], dtype=np.uint64)
    A = _random_sets(rng, n, 60, 0.7)
    B = _random_sets(rng, n, 90, 0.3)
    Ac = _lex_sorted_unique(A ^ full, n)
    got = oracle.mark_supersets(n, Ac, B ^ full)
    want = np.array([any(not np.any(Y & ~X) for X in A) for Y in B])  # Y inside some X
    assert (got == want).all()


def test_mark_supersets_rejects_unsorted_lists():
    n = 8
    # {0} comes before {0, 1}: they first differ at state 1, absent first
    ordered = np.array([[0b01], [0b11]], dtype=np.uint64)
    B = np.array([[0b01], [0b10], [0b11]], dtype=np.uint64)
    assert oracle.mark_supersets(n, ordered, B).tolist() == [True, False, True]
    assert oracle.mark_supersets(n, ordered, B, proper=True).tolist() == [False, False, True]
    with pytest.raises(oracle.OracleError):
        oracle.mark_supersets(n, ordered[::-1].copy(), B)
    with pytest.raises(oracle.OracleError):  # a repeat
        oracle.mark_supersets(n, np.array([[0b01], [0b01]], dtype=np.uint64), B)
    assert oracle.mark_supersets(n, np.zeros((0, 1), np.uint64), B).tolist() == [False, False, False]

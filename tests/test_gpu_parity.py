"""GPU results against the CPU oracle, element by element: r, the least
reset word and every computed level size must be identical (all integer).
Calls go through the C-ABI (Python binding of include/sw.h)."""

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


@pytest.fixture(params=[(0, 0, 0), (0, 4, 0), (0, 0, 64), (1, 0, 0)],
                ids=["bitmap", "bitmap8192", "bitmap_f64", "lop3"])
def meet_algo(sw, request):
    """Runs a test under each meet kernel: vertical bitmaps (default chunk,
    8192-set chunks, and forward tiles of 64 rows so that a level spans many
    tiles), and the direct LOP3 test."""
    old = sw.sw_get_options()
    o = sw.sw_get_options()
    o.meet_algo, o.meet_lane_words, o.meet_f_rows = request.param
    sw.sw_set_options(o)
    yield request.param
    sw.sw_set_options(old)


def resets(delta, word):
    states = np.arange(delta.shape[1])
    for a in word:
        states = delta[a][states]
    return len(np.unique(states)) == 1


def check_sizes(delta, fs, bs):
    assert fs == oracle.level_sizes(delta, 0, len(fs) - 1)
    assert bs == oracle.level_sizes(delta, 1, len(bs) - 1)
    assert len(fs) - 1 + len(bs) - 1 >= 0


def test_hand_examples(sw, ws, meet_algo):
    for ex in json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["examples"]:
        d = np.array(ex["delta"], dtype=np.int32)
        h = sw.load(d)
        r, w = sw.sw_reset_threshold(h, ws=ws)
        assert (r, w) == (ex["r"], ex["word"]), ex["name"]
        fs, bs = sw.sw_level_sizes(h)
        assert fs == ex["fwd_sizes"][: len(fs)] and bs == ex["bwd_sizes"][: len(bs)], ex["name"]
        assert len(fs) + len(bs) - 2 == r


def test_single_random_n40_seed0(sw, ws):
    d = gen.random_automaton(40, 2, 0)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    ro, wo, fo = oracle.forward(d)
    assert (r, w) == (ro, wo)
    fs, bs = sw.sw_level_sizes(h)
    assert fs == fo[: len(fs)]
    check_sizes(d, fs, bs)


@pytest.mark.parametrize("n", list(range(1, 29)))
def test_cerny(sw, ws, meet_algo, n):
    d = gen.cerny(n)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    assert r == (n - 1) ** 2
    assert w == ([] if n == 1 else [1] + ([0] * (n - 1) + [1]) * (n - 2))
    fs, bs = sw.sw_level_sizes(h)
    if n <= 20:
        check_sizes(d, fs, bs)


def _random_cases():
    cases = []
    rng = np.random.default_rng(2024)
    for i in range(60):
        n = int(rng.integers(2, 70))
        k = int(rng.choice([1, 2, 2, 3, 4]))
        cases.append((n, k, 7000 + i))
    return cases


@pytest.mark.parametrize("n,k,seed", _random_cases())
def test_random_vs_oracle(sw, ws, meet_algo, n, k, seed):
    d = gen.random_automaton(n, k, seed)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    ro, wo, fo, bo = oracle.bidir(d)
    assert (r, w) == (ro, wo)
    assert resets(d, w)
    fs, bs = sw.sw_level_sizes(h)
    check_sizes(d, fs, bs)


# Automata whose transitions all land in a scattered core of m states
# (gen.core_automaton): oracle-sized searches whose sets, the backward ones
# above all, spread over W = 4 .. 9 words, with levels of a few thousand sets
# (several 2048-set backward chunks).
CORE_CASES = [(250, 64, 3, 4), (300, 96, 2, 2), (330, 80, 2, 7), (420, 88, 2, 8), (450, 90, 2, 5),
              (520, 72, 2, 6), (576, 80, 2, 3)]


@functools.lru_cache(maxsize=None)
def _core_oracle(n, m, k, seed):
    d = gen.core_automaton(n, m, k, seed)
    r, w, _, _ = oracle.bidir(d)
    return r, tuple(w)


@pytest.mark.parametrize("n,m,k,seed", CORE_CASES)
def test_wide_sets_vs_oracle(sw, ws, meet_algo, n, m, k, seed):
    d = gen.core_automaton(n, m, k, seed)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    ro, wo = _core_oracle(n, m, k, seed)
    assert (r, tuple(w)) == (ro, wo)
    assert resets(d, w)
    fs, bs = sw.sw_level_sizes(h)
    check_sizes(d, fs, bs)


def test_max_letters(sw, ws, meet_algo):
    # k = 255 (the largest alphabet): letter ids up to 254 in the word and
    # candidate ids p*k + a far from powers of two
    for n, seed in ((8, 1), (12, 2)):
        d = gen.random_automaton(n, sw.SW_MAX_LETTERS, seed)
        h = sw.load(d)
        r, w = sw.sw_reset_threshold(h, ws=ws)
        ro, wo, _, _ = oracle.bidir(d)
        assert (r, w) == (ro, wo)
        fs, bs = sw.sw_level_sizes(h)
        check_sizes(d, fs, bs)


def test_ragged_batch_mixed_sizes_and_alphabets(sw, ws):
    # one batch mixing n = 1 .. 130 (one to three words per set) and
    # k = 1 .. 5; every instance must equal its own oracle result
    rng = np.random.default_rng(5)
    ds = [gen.random_automaton(1, 3, 1), gen.random_automaton(4, 1, 2), gen.random_automaton(6, 1, 3)]
    while len(ds) < 40:
        k = int(rng.integers(2, 6))
        n = int(rng.integers(2, 131 if k == 2 else (90 if k == 3 else 60)))
        ds.append(gen.random_automaton(n, k, 900 + len(ds)))
    hs = [sw.load(d) for d in ds]
    rb, wb = sw.sw_batch(hs, ws=ws)
    for i, d in enumerate(ds):
        ro, wo, _, _ = oracle.bidir(d)
        assert (int(rb[i]), wb[i]) == (ro, wo), i
        fs, bs = sw.sw_level_sizes(hs[i])
        check_sizes(d, fs, bs)


def test_batch_equals_single(sw, ws):
    ds = [gen.random_automaton(int(n), 2, 300 + i) for i, n in enumerate([5, 17, 33, 64, 65, 40, 2, 1, 90, 128])]
    hs = [sw.load(d) for d in ds]
    rb, wb = sw.sw_batch(hs, ws=ws)
    sizes_b = [sw.sw_level_sizes(h) for h in hs]
    for i, d in enumerate(ds):
        r, w = sw.sw_reset_threshold(hs[i], ws=ws)
        assert (rb[i], wb[i]) == (r, w)
        ro, wo, _, _ = oracle.bidir(d)
        assert (r, w) == (ro, wo)
        fs, bs = sizes_b[i]
        check_sizes(d, fs, bs)


def test_w_boundaries_and_max_states(sw, ws, meet_algo):
    # n = 64 (Q fills a word), 65 (one bit in a second word), 576 (nine words)
    for n in (63, 64, 65, 128, 129):
        d = gen.random_automaton(n, 2, 11 + n)
        r, w = sw.sw_reset_threshold(sw.load(d), ws=ws)
        assert (r, w) == oracle.bidir(d)[:2]
    n = 576
    halve = np.arange(n) // 2
    perm = np.random.default_rng(1).permutation(n)
    d = np.stack([perm, halve]).astype(np.int32)
    h = sw.load(d)
    r, w = sw.sw_reset_threshold(h, ws=ws)
    ro, wo, fo = oracle.forward(d)
    assert (r, w) == (ro, wo) and r == 10
    fs, bs = sw.sw_level_sizes(h)
    check_sizes(d, fs, bs)


def test_batch_in_waves_equals_roomy_batch(sw, ws):
    # a workspace that holds every instance alone but not all of them at
    # once: instances are set back (their memory freed) and rerun in later
    # waves, and every result must equal the one from a roomy workspace.
    # The smallest size of the list at which every instance fits alone is
    # the one that forces set-backs; smaller ones may fail some instances
    # with SW_ENOMEM, and the rest must still be right.
    ds = gen.batch_random(64, 64, 128, 2, 500)
    hs = [sw.load(d) for d in ds]
    r_big, w_big = sw.sw_batch(hs, ws=ws)
    assert sw.sw_last_stats()["waves"] == 1
    tested = False
    for mib in (16, 24, 32, 48, 64, 96, 128):
        small = sw.workspace(mib << 20)
        r_small, w_small = sw.sw_batch(hs, ws=small, raise_on_error=False)
        st = sw.sw_last_stats()
        ok = r_small >= 0
        assert (r_small[ok] == r_big[ok]).all()
        assert all(w_small[i] == w_big[i] for i in np.nonzero(ok)[0])
        if ok.all():
            assert st["evictions"] > 0 and st["waves"] > 1, (mib, st)
            tested = True
            break
    assert tested
    for i in (0, 17, 63):
        assert (int(r_small[i]), w_small[i]) == oracle.bidir(ds[i])[:2]


def test_word_cap_and_small_workspace(sw, ws):
    d = gen.cerny(6)
    h = sw.load(d)
    with pytest.raises(sw.SwError) as e:
        sw.sw_reset_threshold(h, ws=ws, word_cap=10)
    assert e.value.code == sw.SW_EWORDCAP
    tiny = sw.workspace(300 << 10)
    d = gen.random_automaton(150, 2, 3)
    with pytest.raises(sw.SwError) as e:
        sw.sw_reset_threshold(sw.load(d), ws=tiny)
    assert e.value.code == sw.SW_ENOMEM


def test_batch_device_matches_host_batch(sw, ws):
    import torch
    ds = [gen.random_automaton_ranged(20, 80, 2, s) for s in range(40)]
    ns = [d.shape[1] for d in ds]
    ks = [d.shape[0] for d in ds]
    flat = np.concatenate([d.ravel() for d in ds]).astype(np.int32)
    offs = np.cumsum([0] + [d.size for d in ds[:-1]]).astype(np.int64)
    d_delta = torch.from_numpy(flat).cuda()
    d_r = torch.zeros(len(ds), dtype=torch.int32, device="cuda")
    cap = 256
    word_off = np.arange(len(ds) + 1, dtype=np.int64) * cap
    d_words = torch.zeros(int(word_off[-1]), dtype=torch.uint8, device="cuda")
    rc = sw.sw_batch_device(ns, ks, d_delta, offs, ws=ws, d_r=d_r, d_words=d_words, word_off=word_off)
    assert rc == 0
    rb, wb = sw.sw_batch([sw.load(d) for d in ds], ws=ws)
    r_dev = d_r.cpu().numpy()
    words_dev = d_words.cpu().numpy()
    assert (r_dev == rb).all()
    for i in range(len(ds)):
        assert words_dev[word_off[i]: word_off[i] + r_dev[i]].tolist() == wb[i]


def test_batch_device_not_synchronizing(sw, ws):
    import torch
    good = gen.random_automaton(12, 2, 1)
    bad = np.array([[1, 2, 0], [0, 1, 2]], dtype=np.int32)  # two permutations
    flat = np.concatenate([good.ravel(), bad.ravel()]).astype(np.int32)
    d_delta = torch.from_numpy(flat).cuda()
    d_r = torch.zeros(2, dtype=torch.int32, device="cuda")
    rc = sw.sw_batch_device([12, 3], [2, 2], d_delta, [0, good.size], ws=ws, d_r=d_r)
    assert rc == sw.SW_ENOTSYNC
    r = d_r.cpu().tolist()
    assert r[1] == -1 and r[0] == oracle.forward(good)[0]


def test_server_results_equal_alone(sw):
    """Requests arriving while others run are admitted into the running
    iterations (continuous batching); each result equals the one computed
    alone and the oracle's.  Two long Cerny searches (528 and 729 levels)
    start first, so the later arrivals can only overlap with them if the
    server admits requests mid-run; its counters must show admissions while
    at least two searches were in progress, which a server that ran its
    requests one at a time could not show."""
    import time
    rng = np.random.default_rng(77)
    ds = [gen.cerny(24), gen.cerny(28)]
    for i in range(48):
        k = int(rng.choice([2, 3, 4]))
        n = int(rng.integers(16, {2: 90, 3: 64, 4: 48}[k]))
        ds.append(gen.random_automaton(n, k, 9000 + i))
    ds.append(gen.cerny(12))
    ds.append(np.zeros((2, 1), np.int32))
    want = [oracle.bidir(d)[:2] for d in ds]
    hs = [sw.load(d) for d in ds]
    ws_alone = sw.workspace(256 << 20)
    alone = [sw.sw_reset_threshold(h, ws=ws_alone) for h in hs]
    assert alone == want
    srv = sw.Server(sw.workspace(1 << 30), n_max=128, k_max=4, max_requests=64)
    got = {}
    try:
        for i, h in enumerate(hs):  # staggered arrivals
            while srv.submit(h, i) == sw.SW_EBUSY:
                time.sleep(0.001)
            if i % 5 == 0:
                time.sleep(0.002)
            while (res := srv.poll()) is not None:
                got[res[0]] = res
        t0 = time.time()
        while len(got) < len(hs) and time.time() - t0 < 120:
            res = srv.poll()
            if res is None:
                time.sleep(0.001)
            else:
                got[res[0]] = res
        stats = srv.stats()
    finally:
        srv.close()
    assert len(got) == len(hs)
    for i in range(len(hs)):
        req, r, w, code = got[i]
        assert code == 0 and (r, w) == alone[i] == want[i], i
    assert stats["admitted_while_2"] >= 1, stats
    assert stats["max_active"] >= 3, stats


def test_table_overflow_fails_only_its_instance(sw, ws):
    """A host-side cap on every hash table (sw_options.table_cap_slots, a
    test knob; no device fault) makes the tables of the two large automata
    overflow: those two fail alone with SW_ENOMEM (r = -1), every other
    instance of the same batch is oracle-exact, and without the cap the
    same batch succeeds."""
    small = [gen.random_automaton(int(n), 2, 40 + i) for i, n in enumerate([5, 8, 11, 13, 9, 16, 12, 7, 15, 10])]
    big = [gen.random_automaton(110, 2, 3), gen.random_automaton(120, 2, 4)]
    ds = small[:5] + [big[0]] + small[5:] + [big[1]]
    hs = [sw.load(d) for d in ds]
    old = sw.sw_get_options()
    o = sw.sw_get_options()
    o.table_cap_slots = 2048
    sw.sw_set_options(o)
    try:
        r, w = sw.sw_batch(hs, ws=ws, raise_on_error=False)
        assert sw.lib().sw_last_error() == sw.SW_ENOMEM
    finally:
        sw.sw_set_options(old)
    for i, d in enumerate(ds):
        if d.shape[1] >= 110:
            assert r[i] == -1 and w[i] is None, i
        else:
            assert (int(r[i]), w[i]) == oracle.bidir(d)[:2], i
    r2, w2 = sw.sw_batch(hs, ws=ws)
    for i in (5, len(ds) - 1):
        assert (int(r2[i]), w2[i]) == oracle.bidir(ds[i])[:2]


def test_expmark_direction_rule_same_results(sw, ws):
    """The direction rule of ExpMark estimates (sw_options.dir_rule = 1,
    Section 2.1.2) takes another schedule; r, the word and every level size
    both schedules computed must be the same (they are properties of the
    automaton), and oracle-exact."""
    ds = gen.batch_random(32, 64, 128, 2, 4100)
    hs = [sw.load(d) for d in ds]
    r0, w0 = sw.sw_batch(hs, ws=ws)
    s0 = [sw.sw_level_sizes(h) for h in hs]
    old = sw.sw_get_options()
    o = sw.sw_get_options()
    o.dir_rule = 1
    o.set_cost = 512.0
    sw.sw_set_options(o)
    try:
        r1, w1 = sw.sw_batch(hs, ws=ws)
        s1 = [sw.sw_level_sizes(h) for h in hs]
    finally:
        sw.sw_set_options(old)
    assert (r0 == r1).all() and w0 == w1
    for (f0, b0), (f1, b1) in zip(s0, s1):
        m, mb = min(len(f0), len(f1)), min(len(b0), len(b1))
        assert f0[:m] == f1[:m] and b0[:mb] == b1[:mb]
    for i in (0, 5, 31):
        assert (int(r1[i]), w1[i]) == oracle.bidir(ds[i])[:2]

"""Seeded synthetic automata (the input recipe of the paper's experiments).

This module only makes inputs.  It holds none of the search arithmetic and
is shared, as input, by the GPU library's tests and benchmark and by the
CPU oracle's tests.

Random automata follow Section 3 ("random automaton"): every transition
delta(q, a) is drawn independently and uniformly from Q, and automata that
are not synchronizing are excluded (here: redrawn from the same stream).
The random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), one stream per
instance seed; a 64-bit draw x becomes an integer in [0, m) as
floor(x * m / 2^64) (Lemire's multiply-shift).  SplitMix64 is counter based
(output i depends only on seed + (i + 1) * gamma), so whole blocks of draws
are computed at once with numpy's wrapping uint64 arithmetic.

delta is returned as int32 [k][n], letter-major: delta[a, q] = delta(q, a).
"""

from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_block(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream of `seed`."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def below(x: np.ndarray, m: int) -> np.ndarray:
    """floor(x * m / 2^64) for uint64 x and 0 < m < 2^31, exactly."""
    m64 = np.uint64(m)
    with np.errstate(over="ignore"):
        lo = (x & np.uint64(0xFFFFFFFF)) * m64
        hi = (x >> np.uint64(32)) * m64 + (lo >> np.uint64(32))
    return (hi >> np.uint64(32)).astype(np.int64)


class _Stream:
    def __init__(self, seed: int):
        self.seed = seed
        self.pos = 0

    def draw(self, count: int) -> np.ndarray:
        out = splitmix64_block(self.seed, self.pos, count)
        self.pos += count
        return out


def is_synchronizing(delta: np.ndarray) -> bool:
    """Input filter: every pair of states can be mapped to one state.

    merged[p, q] grows from the diagonal: (p, q) is merged once
    (delta(p, a), delta(q, a)) is merged for some letter a.  Fixed point by
    repeated vectorised gathers.
    """
    delta = np.asarray(delta, dtype=np.int64)
    k, n = delta.shape
    merged = np.eye(n, dtype=bool)
    while True:
        new = merged.copy()
        for a in range(k):
            d = delta[a]
            new |= merged[d[:, None], d[None, :]]
        if new.sum() == merged.sum():
            return bool(merged.all())
        merged = new


def random_automaton(n: int, k: int, seed: int, sink: bool = False) -> np.ndarray:
    """delta(q, a) iid uniform over Q, redrawn until synchronizing.

    With sink=True state 0 is made a sink (delta(0, a) = 0 for every a)
    before the synchronizability filter.
    """
    if n < 1 or k < 1:
        raise ValueError("n and k must be positive")
    st = _Stream(seed)
    while True:
        delta = below(st.draw(k * n), n).reshape(k, n).astype(np.int32)
        if sink:
            delta[:, 0] = 0
        if n == 1 or is_synchronizing(delta):
            return delta


def random_automaton_ranged(n_lo: int, n_hi: int, k: int, seed: int) -> np.ndarray:
    """n drawn first, uniform in [n_lo, n_hi], from the instance's stream;
    then delta as in random_automaton, continuing the same stream."""
    st = _Stream(seed)
    n = n_lo + int(below(st.draw(1), n_hi - n_lo + 1)[0])
    while True:
        delta = below(st.draw(k * n), n).reshape(k, n).astype(np.int32)
        if n == 1 or is_synchronizing(delta):
            return delta


def core_automaton(n: int, m: int, k: int, seed: int) -> np.ndarray:
    """Every transition lands in a core C of m states scattered over Q:
    C is a uniformly random m-subset of Q (the m smallest of n keyed draws),
    and delta(q, a) is uniform over C for every state q, redrawn until
    synchronizing.  After one letter every set lies inside C, so the search
    is as deep as on an m-state automaton, while its sets (backward sets
    above all) still spread over all ceil(n / 64) words."""
    if not 1 <= m <= n or k < 1:
        raise ValueError("need 1 <= m <= n and k >= 1")
    st = _Stream(seed)
    core = np.sort(np.argsort(st.draw(n), kind="stable")[:m])
    while True:
        delta = core[below(st.draw(k * n), m)].reshape(k, n).astype(np.int32)
        if n == 1 or is_synchronizing(delta):
            return delta


def cerny(n: int) -> np.ndarray:
    """The Cerny automaton C_n: letter 0 (a) is the cyclic shift q -> q+1
    mod n, letter 1 (b) maps 0 to 1 and fixes every other state."""
    a = (np.arange(n) + 1) % n
    b = np.arange(n)
    if n >= 2:
        b[0] = 1
    return np.stack([a, b]).astype(np.int32)


def batch_random(count: int, n_lo: int, n_hi: int, k: int, first_seed: int = 0) -> list:
    """`count` ranged random automata with seeds first_seed, first_seed+1, ..."""
    return [random_automaton_ranged(n_lo, n_hi, k, first_seed + i) for i in range(count)]

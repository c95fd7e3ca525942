"""ctypes wrapper of the CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
CPU-baseline leg of the benchmark use it.  The GPU library never imports it.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ERRORS = {
    0: "ok",
    -1: "invalid arguments",
    -2: "too many sets",
    -3: "not synchronizing",
    -4: "word does not fit",
    -5: "out of host memory",
    -6: "no reset word up to max_len",
}


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc -O3 (portable: no -march, so that it
    builds and gives the same results on x86 and Arm hosts)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        lib.oracle_brute.argtypes = [ctypes.c_int, ctypes.c_int, p, ctypes.c_int, p, p]
        lib.oracle_forward.argtypes = [ctypes.c_int, ctypes.c_int, p, i64, p, p, i32, p, i32, p]
        lib.oracle_level_sizes.argtypes = [ctypes.c_int, ctypes.c_int, p, ctypes.c_int, i32, i64, p]
        lib.oracle_bidir.argtypes = [ctypes.c_int, ctypes.c_int, p, i64, p, p, i32, p, p, p, p, i32]
        lib.oracle_is_synchronizing.argtypes = [ctypes.c_int, ctypes.c_int, p]
        lib.oracle_reduced_level_sizes.argtypes = [ctypes.c_int, ctypes.c_int, p, ctypes.c_int, i32, i64, p]
        lib.oracle_bidir_reduced.argtypes = [ctypes.c_int, ctypes.c_int, p, i64, i32, i32, p, p, i32, p, p, p, p, i32]
        lib.oracle_beam.argtypes = [ctypes.c_int, ctypes.c_int, p, i64, i32, p, p, i32, p, i32, p]
        lib.oracle_inverse_dfs_r.argtypes = [ctypes.c_int, ctypes.c_int, p, i32, i32, i32, i32, i64, p]
        lib.oracle_mark_supersets.argtypes = [ctypes.c_int, p, i64, p, i64, ctypes.c_int, i32, p]
        lib.oracle_mark_supersets.restype = i64
        lib.oracle_beam.restype = ctypes.c_int
        for f in (lib.oracle_brute, lib.oracle_forward, lib.oracle_level_sizes, lib.oracle_bidir,
                  lib.oracle_is_synchronizing, lib.oracle_reduced_level_sizes, lib.oracle_bidir_reduced):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _delta(delta):
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.int32))
    if d.ndim != 2:
        raise ValueError("delta must be [k][n]")
    return d, d.shape[1], d.shape[0]


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def brute(delta, max_len: int = 24):
    """O0: (r, word) by enumerating words in length-lexicographic order."""
    d, n, k = _delta(delta)
    r = np.zeros(1, np.int32)
    w = np.zeros(64, np.uint8)
    rc = _load().oracle_brute(n, k, _ptr(d), max_len, _ptr(r), _ptr(w))
    if rc:
        raise OracleError(rc, "oracle_brute")
    return int(r[0]), w[: r[0]].tolist()


def forward(delta, max_sets: int = 50_000_000, word_cap: int = 1 << 20):
    """O1: (r, word, level_sizes) by forward BFS over the power automaton."""
    d, n, k = _delta(delta)
    r = np.zeros(1, np.int32)
    w = np.zeros(word_cap, np.uint8)
    sizes = np.zeros(word_cap + 1, np.int64)
    nl = np.zeros(1, np.int32)
    rc = _load().oracle_forward(n, k, _ptr(d), max_sets, _ptr(r), _ptr(w), word_cap, _ptr(sizes),
                                len(sizes), _ptr(nl))
    if rc:
        raise OracleError(rc, "oracle_forward")
    return int(r[0]), w[: r[0]].tolist(), sizes[: nl[0]].tolist()


def level_sizes(delta, direction: int, depth: int, max_sets: int = 50_000_000):
    """Sizes of deduplicated levels 0..depth: direction 0 = images of Q,
    1 = preimages of singletons."""
    d, n, k = _delta(delta)
    sizes = np.zeros(depth + 1, np.int64)
    rc = _load().oracle_level_sizes(n, k, _ptr(d), direction, depth, max_sets, _ptr(sizes))
    if rc:
        raise OracleError(rc, "oracle_level_sizes")
    return sizes.tolist()


def bidir(delta, max_sets: int = 50_000_000, word_cap: int = 1 << 20):
    """O2: (r, word, fwd_sizes, bwd_sizes) by bidirectional BFS (Alg. 1,
    duplicate deletion and equality history only)."""
    d, n, k = _delta(delta)
    r = np.zeros(1, np.int32)
    w = np.zeros(word_cap, np.uint8)
    cap = 4096
    fs = np.zeros(cap, np.int64)
    bs = np.zeros(cap, np.int64)
    nf = np.zeros(1, np.int32)
    nb = np.zeros(1, np.int32)
    rc = _load().oracle_bidir(n, k, _ptr(d), max_sets, _ptr(r), _ptr(w), word_cap, _ptr(fs), _ptr(nf),
                              _ptr(bs), _ptr(nb), cap)
    if rc:
        raise OracleError(rc, "oracle_bidir")
    return int(r[0]), w[: r[0]].tolist(), fs[: nf[0]].tolist(), bs[: nb[0]].tolist()


def reduced_level_sizes(delta, direction: int, depth: int, max_sets: int = 50_000_000):
    """Sizes of the levels 0..depth of one direction under the inclusion
    reductions of Alg. 1: 0 = images of Q (minimal sets; supersets of
    earlier levels removed), 1 = preimages of singletons (maximal sets;
    subsets of earlier levels removed)."""
    d, n, k = _delta(delta)
    sizes = np.zeros(depth + 1, np.int64)
    rc = _load().oracle_reduced_level_sizes(n, k, _ptr(d), direction, depth, max_sets, _ptr(sizes))
    if rc:
        raise OracleError(rc, "oracle_reduced_level_sizes")
    return sizes.tolist()


def bidir_reduced(delta, fwd_depth: int = -1, dirs: int = 3, max_sets: int = 50_000_000,
                  word_cap: int = 1 << 20):
    """O3: (r, word, fwd_sizes, bwd_sizes) by Alg. 1 with the inclusion
    reductions.  fwd_depth >= 0 fixes the forward depth of the meet (the
    word depends on it; r and the sizes do not).  dirs: 1 reduces the BFS
    side only, 2 the IBFS side only, 3 both; an unreduced side keeps the
    equality history."""
    d, n, k = _delta(delta)
    r = np.zeros(1, np.int32)
    w = np.zeros(word_cap, np.uint8)
    cap = 4096
    fs = np.zeros(cap, np.int64)
    bs = np.zeros(cap, np.int64)
    nf = np.zeros(1, np.int32)
    nb = np.zeros(1, np.int32)
    rc = _load().oracle_bidir_reduced(n, k, _ptr(d), max_sets, fwd_depth, dirs, _ptr(r), _ptr(w), word_cap,
                                      _ptr(fs), _ptr(nf), _ptr(bs), _ptr(nb), cap)
    if rc:
        raise OracleError(rc, "oracle_bidir_reduced")
    return int(r[0]), w[: r[0]].tolist(), fs[: nf[0]].tolist(), bs[: nb[0]].tolist()


def beam(delta, beam_size: int, max_depth: int = 1 << 16):
    """O4: (R, word, level_sizes) of the cut-off inverse BFS that keeps the
    beam_size largest preimages of every depth; R >= r."""
    d, n, k = _delta(delta)
    r = np.zeros(1, np.int32)
    w = np.zeros(max_depth + 1, np.uint8)
    sizes = np.zeros(max_depth + 1, np.int64)
    nl = np.zeros(1, np.int32)
    rc = _load().oracle_beam(n, k, _ptr(d), beam_size, max_depth, _ptr(r), _ptr(w), len(w), _ptr(sizes), len(sizes),
                             _ptr(nl))
    if rc:
        raise OracleError(rc, "oracle_beam")
    return int(r[0]), w[: r[0]].tolist(), sizes[: nl[0]].tolist()


def inverse_dfs_r(delta, fwd_depth: int, bwd_depth: int, dirs: int = 0, max_depth: int = 24,
                  max_sets: int = 50_000_000) -> int:
    """O5: r from the BFS level at fwd_depth and the IBFS level at bwd_depth
    by the inverse DFS phase of Section 2.2 (depth-first over preimages, no
    history, brute-force subset checks against the BFS level).  dirs: bit 0
    reduces the BFS side, bit 1 the IBFS side (Alg. 1's inclusion
    reductions, as bidir_reduced)."""
    d, n, k = _delta(delta)
    r = np.zeros(1, np.int32)
    rc = _load().oracle_inverse_dfs_r(n, k, _ptr(d), fwd_depth, bwd_depth, dirs, max_depth, max_sets, _ptr(r))
    if rc:
        raise OracleError(rc, "oracle_inverse_dfs_r")
    return int(r[0])


def mark_supersets(n: int, A, B, proper: bool = False, min_brute: int = 4):
    """O6, Alg. 2: boolean marks of the sets of B (uint64 [nb][W] bitsets)
    that contain (properly, when proper) some set of A (uint64 [na][W],
    sorted lexicographically from state 0, absent before present, no
    repeats)."""
    W = (n + 63) // 64
    A = np.ascontiguousarray(np.asarray(A, dtype=np.uint64).reshape(-1, W))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.uint64).reshape(-1, W))
    marks = np.zeros(max(len(B), 1), np.uint8)
    rc = _load().oracle_mark_supersets(n, _ptr(A), len(A), _ptr(B), len(B), int(bool(proper)), min_brute,
                                       _ptr(marks))
    if rc < 0:
        raise OracleError(int(rc), "oracle_mark_supersets")
    return marks[: len(B)].astype(bool)


def is_synchronizing(delta) -> bool:
    d, n, k = _delta(delta)
    rc = _load().oracle_is_synchronizing(n, k, _ptr(d))
    if rc < 0:
        raise OracleError(rc, "oracle_is_synchronizing")
    return bool(rc)

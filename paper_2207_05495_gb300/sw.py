"""Python binding of the C-ABI in include/sw.h (argument marshalling only).

Every step of the search runs in the CUDA library libsw.so; this module only
converts arguments, supplies device workspace and streams from PyTorch, and
turns status codes into exceptions.  If the library is missing it raises; it
has no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsw.so")
_lib = None

SW_OK, SW_EINVAL, SW_ENOTSYNC, SW_ENOMEM, SW_ETIMEOUT, SW_EWORDCAP, SW_ECUDA, SW_EBUSY, SW_EAGAIN, \
    SW_EINTERNAL, SW_ENOTFOUND = range(11)
SW_MAX_STATES = 576
SW_BEAM_MAX_STATES = 8192
SW_MAX_LETTERS = 255


class SwError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().sw_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class sw_options(ctypes.Structure):
    _fields_ = [("meet_algo", ctypes.c_int32), ("meet_rows_per_thread", ctypes.c_int32),
                ("meet_b_tile", ctypes.c_int32), ("meet_f_rows", ctypes.c_int32),
                ("meet_lane_words", ctypes.c_int32),
                ("dir_theta", ctypes.c_double), ("set_cost", ctypes.c_double), ("reduce", ctypes.c_int32),
                ("table_cap_slots", ctypes.c_int32), ("dir_rule", ctypes.c_int32), ("dfs_sets", ctypes.c_int64)]


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"CUDA library {_LIB_PATH} is missing: build it with "
                               "paper_2207_05495_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(_LIB_PATH)
        p, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        L.sw_load_automaton.argtypes = [i32, i32, p]
        L.sw_load_automaton.restype = p
        L.sw_free.argtypes = [p]
        L.sw_free.restype = None
        L.sw_last_error.restype = i32
        L.sw_error_string.argtypes = [i32]
        L.sw_error_string.restype = ctypes.c_char_p
        L.sw_workspace_min_bytes.argtypes = [i32, i32, i32]
        L.sw_workspace_min_bytes.restype = sz
        L.sw_reset_threshold.argtypes = [p, p, p, sz, p, p, i32]
        L.sw_reset_threshold.restype = i32
        L.sw_level_sizes.argtypes = [p, p, i32, p, p, i32, p]
        L.sw_level_sizes.restype = i32
        L.sw_batch.argtypes = [p, i32, p, p, sz, p, p, p, i64]
        L.sw_batch.restype = i32
        L.sw_batch_device.argtypes = [i32, p, p, p, p, p, p, sz, p, p, p, i64]
        L.sw_batch_device.restype = i32
        L.sw_last_stats.argtypes = [p] * 19
        L.sw_last_stats.restype = i32
        L.sw_beam.argtypes = [i32, i32, p, p, p, sz, i64, i32, p, p, i32]
        L.sw_beam.restype = i32
        L.sw_expmark.argtypes = [ctypes.c_double] * 4
        L.sw_expmark.restype = ctypes.c_double
        L.sw_probe_int_peak.argtypes = [p, p, sz, p]
        L.sw_probe_int_peak.restype = i32
        L.sw_last_reduce_stats.argtypes = [p, p, p, p]
        L.sw_last_reduce_stats.restype = i32
        L.sw_last_host_stats.argtypes = [p] * 5
        L.sw_last_host_stats.restype = i32
        L.sw_last_dfs_stats.argtypes = [p] * 3
        L.sw_last_dfs_stats.restype = i32
        L.sw_set_timing.argtypes = [i32]
        L.sw_set_timing.restype = None
        L.sw_get_options.argtypes = [p]
        L.sw_get_options.restype = None
        L.sw_set_options.argtypes = [p]
        L.sw_set_options.restype = None
        L.sw_reset_threshold_static.argtypes = [p, p, p, p, i32]
        L.sw_reset_threshold_static.restype = i32
        L.sw_server_create.argtypes = [p, sz, i32, i32, i32, i32, p, p]
        L.sw_server_create.restype = i32
        L.sw_server_submit.argtypes = [p, p, ctypes.c_uint64]
        L.sw_server_submit.restype = i32
        L.sw_server_poll.argtypes = [p, p, p, p, i32, p]
        L.sw_server_poll.restype = i32
        L.sw_server_pending.argtypes = [p, p, p, p]
        L.sw_server_pending.restype = i32
        L.sw_server_stats.argtypes = [p, p, p, p, p, p]
        L.sw_server_stats.restype = i32
        L.sw_server_destroy.argtypes = [p]
        L.sw_server_destroy.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Automaton:
    """An owned sw_handle (freed with the object)."""

    def __init__(self, ptr: int, n: int, k: int):
        self.ptr, self.n, self.k = ptr, n, k

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.sw_free(ctypes.c_void_p(self.ptr))
            self.ptr = None


def sw_load_automaton(n: int, k: int, delta) -> Automaton:
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.int32))
    if d.shape != (k, n):
        raise ValueError(f"delta must have shape (k, n) = ({k}, {n})")
    h = lib().sw_load_automaton(n, k, _ptr(d))
    if not h:
        raise SwError(lib().sw_last_error(), "sw_load_automaton")
    return Automaton(h, n, k)


def load(delta) -> Automaton:
    """sw_load_automaton for a [k][n] array."""
    d = np.asarray(delta)
    return sw_load_automaton(d.shape[1], d.shape[0], d)


def workspace(nbytes: int):
    """Device workspace from PyTorch's allocator (256-byte aligned)."""
    import torch
    return torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")


def _ws_args(ws):
    return ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(ws.numel())


def sw_workspace_min_bytes(n_max: int, k_max: int, count: int) -> int:
    return int(lib().sw_workspace_min_bytes(n_max, k_max, count))


def sw_reset_threshold(h: Automaton, stream=None, ws=None, word_cap: int = 1 << 16):
    """(r, word) of one automaton.  ws: a device uint8 tensor (default: 256 MiB)."""
    if ws is None:
        ws = workspace(256 << 20)
    r = np.zeros(1, np.int32)
    word = np.zeros(max(word_cap, 1), np.uint8)
    p, nb = _ws_args(ws)
    rc = lib().sw_reset_threshold(ctypes.c_void_p(h.ptr), _stream(stream), p, nb, _ptr(r), _ptr(word), word_cap)
    if rc != SW_OK:
        raise SwError(rc, "sw_reset_threshold")
    return int(r[0]), word[: r[0]].tolist()


def sw_reset_threshold_static(h: Automaton, stream=None, word_cap: int = 1 << 16):
    """(r, word) of one automaton without any device allocation: the search
    runs in the library's fixed 64 MiB device scratch (see include/sw.h).
    Calls must not overlap on the GPU."""
    r = np.zeros(1, np.int32)
    word = np.zeros(max(word_cap, 1), np.uint8)
    rc = lib().sw_reset_threshold_static(ctypes.c_void_p(h.ptr), _stream(stream), _ptr(r), _ptr(word), word_cap)
    if rc != SW_OK:
        raise SwError(rc, "sw_reset_threshold_static")
    return int(r[0]), word[: r[0]].tolist()


def sw_beam(delta, beam: int, stream=None, ws=None, max_depth: int = 1 << 16):
    """(R, word) of the cut-off inverse BFS keeping the `beam` largest
    preimages of every depth (an upper bound R >= r).  delta: [k][n] int32
    array, n up to SW_BEAM_MAX_STATES."""
    d = np.ascontiguousarray(np.asarray(delta, dtype=np.int32))
    k, n = d.shape
    if ws is None:
        ws = workspace(1 << 30)
    R = np.zeros(1, np.int32)
    word = np.zeros(max(max_depth, 1), np.uint8)
    p, nb = _ws_args(ws)
    rc = lib().sw_beam(n, k, _ptr(d), _stream(stream), p, nb, beam, max_depth, _ptr(R), _ptr(word), len(word))
    if rc != SW_OK:
        raise SwError(rc, "sw_beam")
    return int(R[0]), word[: R[0]].tolist()


def sw_level_sizes(h: Automaton, cap: int = 1 << 16):
    """(forward sizes, backward sizes) of the last search of h."""
    f = np.zeros(cap, np.int64)
    b = np.zeros(cap, np.int64)
    nf = np.zeros(1, np.int32)
    nbk = np.zeros(1, np.int32)
    rc = lib().sw_level_sizes(ctypes.c_void_p(h.ptr), _ptr(f), cap, _ptr(nf), _ptr(b), cap, _ptr(nbk))
    if rc != SW_OK:
        raise SwError(rc, "sw_level_sizes")
    return f[: nf[0]].tolist(), b[: nbk[0]].tolist()


def sw_batch(hs, stream=None, ws=None, word_cap: int = 4096, raise_on_error: bool = True):
    """(r array, list of words) for a list of Automaton handles."""
    count = len(hs)
    arr = (ctypes.c_void_p * count)(*[h.ptr for h in hs])
    r = np.zeros(count, np.int32)
    off = np.arange(count + 1, dtype=np.int64) * word_cap
    words = np.zeros(max(int(off[-1]), 1), np.uint8)
    if ws is None:
        ws = workspace(1 << 30)
    p, nb = _ws_args(ws)
    rc = lib().sw_batch(arr, count, _stream(stream), p, nb, _ptr(r), _ptr(words), _ptr(off), int(off[-1]))
    if rc != SW_OK and raise_on_error:
        raise SwError(rc, "sw_batch")
    out = [words[off[i]: off[i] + r[i]].tolist() if r[i] >= 0 else None for i in range(count)]
    return r, out


def sw_batch_device(n, k, d_delta, delta_off, stream=None, ws=None, d_r=None, d_words=None, word_off=None):
    """Device-resident batch: d_delta, d_r, d_words are CUDA tensors
    (int32, int32, uint8); n, k, delta_off, word_off host arrays.  Returns
    the status code (0 = every instance succeeded)."""
    n = np.ascontiguousarray(n, dtype=np.int32)
    k = np.ascontiguousarray(k, dtype=np.int32)
    delta_off = np.ascontiguousarray(delta_off, dtype=np.int64)
    count = len(n)
    p, nb = _ws_args(ws)
    if d_words is not None:
        word_off = np.ascontiguousarray(word_off, dtype=np.int64)
        wptr, woff, wcap = ctypes.c_void_p(d_words.data_ptr()), _ptr(word_off), int(word_off[-1])
    else:
        wptr, woff, wcap = None, None, 0
    return int(lib().sw_batch_device(count, _ptr(n), _ptr(k), ctypes.c_void_p(d_delta.data_ptr()),
                                     _ptr(delta_off), _stream(stream), p, nb,
                                     ctypes.c_void_p(d_r.data_ptr()), wptr, woff, wcap))


def sw_last_stats() -> dict:
    """Counters of the calling thread's last search (sw_last_stats), with
    the marking kernel's (sw_last_reduce_stats) under the keys mark_* and
    the time between kernels (sw_last_host_stats)."""
    d = _last_stats()
    d.update(sw_last_reduce_stats())
    d.update(sw_last_host_stats())
    d.update(sw_last_dfs_stats())
    return d


def _last_stats() -> dict:
    pairs, cand, launches, peak = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    iters, rows = ctypes.c_int64(), ctypes.c_int64()
    wms, rms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    sel, upd = ctypes.c_double(), ctypes.c_double()
    it, ml, wv, ev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    mm, em, cm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lw = ctypes.c_int32()
    lib().sw_last_stats(ctypes.byref(pairs), ctypes.byref(cand), ctypes.byref(it), ctypes.byref(mm),
                        ctypes.byref(em), ctypes.byref(cm), ctypes.byref(ml), ctypes.byref(launches),
                        ctypes.byref(wv), ctypes.byref(ev), ctypes.byref(peak), ctypes.byref(iters),
                        ctypes.byref(rows), ctypes.byref(wms), ctypes.byref(rms), ctypes.byref(sms),
                        ctypes.byref(sel), ctypes.byref(upd), ctypes.byref(lw))
    return {"pairs": pairs.value, "candidates": cand.value, "iterations": it.value, "meet_ms": mm.value,
            "expand_ms": em.value, "compact_ms": cm.value, "meet_launches": ml.value,
            "launches": launches.value, "waves": wv.value, "evictions": ev.value, "arena_peak": peak.value,
            "and_iters": iters.value, "rows_transposed": rows.value, "words_ms": wms.value,
            "run_ms": rms.value, "sync_ms": sms.value, "select_ms": sel.value, "update_ms": upd.value,
            "meet_lane_words": lw.value}


def sw_last_host_stats() -> dict:
    v = [ctypes.c_double() for _ in range(5)]
    lib().sw_last_host_stats(*[ctypes.byref(x) for x in v])
    return dict(zip(("stage_ms", "plan_ms", "post_ms", "table_ms", "gap_ms"), (x.value for x in v)))


def sw_last_dfs_stats() -> dict:
    v = [ctypes.c_int64() for _ in range(3)]
    lib().sw_last_dfs_stats(*[ctypes.byref(x) for x in v])
    return dict(zip(("dfs_instances", "dfs_chunks", "dfs_sets"), (x.value for x in v)))


def sw_last_reduce_stats() -> dict:
    ms, pairs, steps, rows = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib().sw_last_reduce_stats(ctypes.byref(ms), ctypes.byref(pairs), ctypes.byref(steps), ctypes.byref(rows))
    return {"mark_ms": ms.value, "mark_pairs": pairs.value, "mark_steps": steps.value, "mark_rows": rows.value}


def sw_expmark(a_s: float, b_s: float, a_d: float, b_d: float) -> float:
    """ExpMark of Section 2.1.2 (host computation in the library)."""
    return float(lib().sw_expmark(a_s, b_s, a_d, b_d))


def sw_probe_int_peak(stream=None) -> float:
    """LOP3 results retired per SM clock (sw_probe_int_peak)."""
    ws = workspace(1 << 20)
    v = ctypes.c_double()
    p, nb = _ws_args(ws)
    rc = lib().sw_probe_int_peak(_stream(stream), p, nb, ctypes.byref(v))
    if rc != SW_OK:
        raise SwError(rc, "sw_probe_int_peak")
    return v.value


def sw_set_timing(on: bool) -> None:
    lib().sw_set_timing(1 if on else 0)


def sw_get_options() -> sw_options:
    o = sw_options()
    lib().sw_get_options(ctypes.byref(o))
    return o


def sw_set_options(o: sw_options) -> None:
    lib().sw_set_options(ctypes.byref(o))


class Server:
    """sw_server_*: continuous batching of searches on one stream."""

    def __init__(self, ws, n_max: int, k_max: int, max_requests: int = 4096, word_cap: int = 4096, stream=None):
        self.ws = ws  # kept alive for the server's lifetime
        self.word_cap = word_cap
        self._word = np.zeros(word_cap, np.uint8)
        srv = ctypes.c_void_p()
        p, nb = _ws_args(ws)
        rc = lib().sw_server_create(p, nb, n_max, k_max, max_requests, word_cap, _stream(stream),
                                    ctypes.byref(srv))
        if rc != SW_OK:
            raise SwError(rc, "sw_server_create")
        self.ptr = srv.value

    def submit(self, h: Automaton, req_id: int) -> int:
        """SW_OK, or SW_EBUSY when the submission queue is full."""
        rc = lib().sw_server_submit(ctypes.c_void_p(self.ptr), ctypes.c_void_p(h.ptr), req_id)
        if rc not in (SW_OK, SW_EBUSY):
            raise SwError(rc, "sw_server_submit")
        return rc

    def poll(self):
        """(req_id, r, word, code) of a finished request, or None."""
        req = ctypes.c_uint64()
        r = ctypes.c_int32()
        code = ctypes.c_int32()
        rc = lib().sw_server_poll(ctypes.c_void_p(self.ptr), ctypes.byref(req), ctypes.byref(r), _ptr(self._word),
                                  self.word_cap, ctypes.byref(code))
        if rc == SW_EAGAIN:
            return None
        if rc != SW_OK:
            raise SwError(rc, "sw_server_poll")
        word = self._word[: r.value].tolist() if code.value == SW_OK else None
        return req.value, r.value, word, code.value

    def pending(self):
        q, a, f = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        rc = lib().sw_server_pending(ctypes.c_void_p(self.ptr), ctypes.byref(q), ctypes.byref(a), ctypes.byref(f))
        if rc != SW_OK:
            raise SwError(rc, "sw_server_pending")
        return q.value, a.value, f.value

    def stats(self) -> dict:
        a, a1, a2, it = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        mx = ctypes.c_int32()
        rc = lib().sw_server_stats(ctypes.c_void_p(self.ptr), ctypes.byref(a), ctypes.byref(a1), ctypes.byref(a2),
                                   ctypes.byref(mx), ctypes.byref(it))
        if rc != SW_OK:
            raise SwError(rc, "sw_server_stats")
        return {"admitted": a.value, "admitted_while_1": a1.value, "admitted_while_2": a2.value,
                "max_active": mx.value, "iterations": it.value}

    def close(self):
        if getattr(self, "ptr", None):
            lib().sw_server_destroy(ctypes.c_void_p(self.ptr))
            self.ptr = None

    def __del__(self):
        self.close()

"""The C-ABI library builds, loads and exports every declared entry point;
its host-side validation works without a GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2207_05495_gb300 import build, gen, sw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sw_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sw.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "sw_reset_threshold" in names and "sw_batch" in names
    raw = ctypes.CDLL(build.LIB)
    for name in names:
        assert hasattr(raw, name), name


def test_error_strings(lib):
    assert lib.sw_error_string(0) == b"ok"
    assert b"not synchronizing" in lib.sw_error_string(2)


def test_load_validates_without_gpu(lib):
    d = gen.random_automaton(20, 2, 1)
    h = sw.load(d)
    assert h.n == 20 and h.k == 2
    with pytest.raises(sw.SwError) as e:
        sw.load(np.array([[1, 0], [0, 1]], dtype=np.int32))  # two permutations
    assert e.value.code == sw.SW_ENOTSYNC
    with pytest.raises(sw.SwError) as e:
        sw.load(np.array([[0, 2]], dtype=np.int32))
    assert e.value.code == sw.SW_EINVAL
    with pytest.raises(sw.SwError) as e:
        sw.sw_load_automaton(sw.SW_MAX_STATES + 1, 1, np.zeros((1, sw.SW_MAX_STATES + 1), np.int32))
    assert e.value.code == sw.SW_EINVAL
    with pytest.raises(sw.SwError) as e:
        sw.sw_level_sizes(h)  # never searched
    assert e.value.code == sw.SW_EINVAL


def test_load_agrees_with_generator_filter(lib):
    rng = np.random.default_rng(5)
    for _ in range(300):
        n = int(rng.integers(2, 9))
        d = rng.integers(0, n, size=(2, n)).astype(np.int32)
        ok = gen.is_synchronizing(d)
        if ok:
            sw.load(d)
        else:
            with pytest.raises(sw.SwError):
                sw.load(d)


def test_workspace_min_bytes(lib):
    a = sw.sw_workspace_min_bytes(40, 2, 1)
    b = sw.sw_workspace_min_bytes(192, 2, 4096)
    assert 0 < a < b
    assert sw.sw_workspace_min_bytes(0, 2, 1) == 0


def test_options_roundtrip(lib):
    o = sw.sw_get_options()
    assert o.dir_theta == 1.0 and o.set_cost == 8192.0 and o.meet_f_rows == 4096
    o.dir_theta = -3.0  # invalid: reset to the default
    sw.sw_set_options(o)
    assert sw.sw_get_options().dir_theta == 1.0


def test_expmark_cost_estimate(lib):
    # Section 2.1.2's ExpMark on the host (no GPU): a value worked out by
    # hand (w = 1.5 / 0.95, exponent ln 1.5 / ln w = 0.8877, 1000^0.8877 =
    # 460.4, factor 1.5 / 0.5 + 1 / (0.1 - 0.05) = 23), linear in Bs,
    # increasing in As, and close to linear in As for very sparse A lists
    v = sw.sw_expmark(1000, 1000, 0.1, 0.5)
    assert abs(v / (1000 * 23 * 460.4) - 1) < 1e-3
    assert abs(sw.sw_expmark(1000, 2000, 0.1, 0.5) / v - 2) < 1e-9
    assert sw.sw_expmark(2000, 1000, 0.1, 0.5) > v
    sparse = sw.sw_expmark(1e6, 10, 1e-6, 0.5) / sw.sw_expmark(1e5, 10, 1e-6, 0.5)
    assert 9.9 < sparse < 10.0
    assert sw.sw_expmark(0, 10, 0.1, 0.5) == 0.0


def test_options_round_trip_and_clamp(lib):
    # the struct layout matches the library's (the last field survives a
    # round trip) and out-of-range values are clamped on the host
    old = sw.sw_get_options()
    try:
        o = sw.sw_get_options()
        o.dfs_sets = 12345
        o.dir_rule = 1
        sw.sw_set_options(o)
        got = sw.sw_get_options()
        assert (got.dfs_sets, got.dir_rule) == (12345, 1)
        o.dfs_sets = -7
        o.reduce = 9
        sw.sw_set_options(o)
        got = sw.sw_get_options()
        assert (got.dfs_sets, got.reduce) == (0, 0)
        o.dfs_sets = -1
        sw.sw_set_options(o)
        assert sw.sw_get_options().dfs_sets == -1
    finally:
        sw.sw_set_options(old)


def test_every_declaration_is_documented():
    # each entry point of the header has a comment block (what it computes,
    # with the paper's passage where one applies, and argument layout,
    # ownership and errors) ending at most 25 lines above its declaration;
    # a block may serve a group of declarations, a typedef or a #define
    text = open(os.path.join(ROOT, "include", "sw.h")).read()
    lines = text.splitlines()
    in_comment = False
    undocumented = []
    last_comment_end = -10**9
    for i, line in enumerate(lines):
        st = line.strip()
        if st.startswith("/*"):
            in_comment = True
        if in_comment:
            if st.endswith("*/"):
                in_comment = False
                last_comment_end = i
            continue
        m = re.match(r"^[A-Za-z_][\w\s\*]*?\b(sw_[a-z_]+)\s*\(", line)
        if m and i - last_comment_end > 25:
            undocumented.append(m.group(1))
    assert not undocumented, undocumented

"""The full 4096-automaton workload (n uniform in [64, 192], k = 2, seeds
0..4095) in the launch configuration the benchmark times (sw_batch_device
with the automata in device memory, and sw_batch with host buffers).

Sampled outputs are compared with stored oracle values
(tests/golden/c3_sample.json, written by tests/golden/make_golden.py from
oracle.bidir alone): r and the least word must be identical.  For every
instance the word must reset Q, have length r, and r must respect the
Frankl-Pin bound; both entry points must agree everywhere; level sizes of
the smaller sampled instances must equal the oracle's."""

import json
import os

import numpy as np
import pytest

import oracle
from paper_2207_05495_gb300 import gen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c3_sample.json")


@pytest.fixture(scope="module")
def sw():
    import torch
    assert torch.cuda.is_available()
    from paper_2207_05495_gb300 import build, sw as swmod
    build.build()
    return swmod


def test_c3_full_batch(sw):
    import torch
    ds = gen.batch_random(4096, 64, 192, 2, 0)
    ns = np.array([d.shape[1] for d in ds], np.int32)
    ks = np.array([d.shape[0] for d in ds], np.int32)
    flat = np.concatenate([d.ravel() for d in ds]).astype(np.int32)
    offs = np.concatenate([[0], np.cumsum([d.size for d in ds])[:-1]]).astype(np.int64)
    cap = 1024
    word_off = np.arange(len(ds) + 1, dtype=np.int64) * cap
    ws = sw.workspace(160 << 30)
    d_delta = torch.from_numpy(flat).cuda()
    d_r = torch.zeros(len(ds), dtype=torch.int32, device="cuda")
    d_words = torch.zeros(int(word_off[-1]), dtype=torch.uint8, device="cuda")
    assert sw.sw_batch_device(ns, ks, d_delta, offs, ws=ws, d_r=d_r, d_words=d_words, word_off=word_off) == 0
    r = d_r.cpu().numpy()
    words = d_words.cpu().numpy()
    hs = [sw.load(d) for d in ds]
    rh, wh = sw.sw_batch(hs, ws=ws, word_cap=cap)
    assert (rh == r).all()
    for i, d in enumerate(ds):
        w = words[word_off[i]: word_off[i] + r[i]].tolist()
        assert w == wh[i]
        st = np.arange(d.shape[1])
        for a in w:
            st = d[a][st]
        assert len(np.unique(st)) == 1, i
        n = d.shape[1]
        assert 0 < r[i] <= (n ** 3 - n) // 6
    gold = json.load(open(GOLDEN))
    assert len(gold["instances"]) >= 60
    for e in gold["instances"]:
        i = e["seed"]
        assert (int(r[i]), wh[i]) == (e["r"], e["word"]), i
        if e["n"] <= 96:
            fs, bs = sw.sw_level_sizes(hs[i])
            assert fs == oracle.level_sizes(ds[i], 0, len(fs) - 1)
            assert bs == oracle.level_sizes(ds[i], 1, len(bs) - 1)

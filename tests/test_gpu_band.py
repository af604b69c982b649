"""Sakoe-Chiba band (Table I) on the GPU against the CPU oracle: costs, |pi|,
paths and DBA prototypes bit-exact to the FP32 mirror, for bands from the
narrowest accepted one to no restriction, uneven lengths in both directions,
several row bands with a ragged last one, and checkpointed codes."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2404_12134_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wts():
    from paper_2404_12134_gb300 import api
    return api


def _pack(cyc):
    offs = np.concatenate([[0], np.cumsum([len(c) for c in cyc])]).astype(np.int64)
    return np.ascontiguousarray(np.concatenate(cyc).astype(np.float32)), offs


def _narrowest(M, lengths):
    """The smallest band accepted for every pair (floor(w M N) >= max(M, N))."""
    w = max(max(M, n) / (M * n) for n in lengths)
    while any(math.floor(w * M * n) < max(M, n) for n in lengths):
        w = math.nextafter(w, 2.0)
    return w


@pytest.mark.parametrize("M,lengths,d", [
    (700, [700, 350, 1400, 5], 2),            # N = M, N < M, N > M, very short
    (1300, [1000, 2100, 1299, 640], 3),       # three row bands, ragged
    (37, [90, 37, 12], 1),
])
def test_banded_dtw_bit_exact(wts, M, lengths, d):
    rng = np.random.default_rng(300 + M)
    B = rng.normal(size=(M, d)).astype(np.float32)
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in lengths]
    data, offs = _pack(cyc)
    gb = wts.Batch.from_numpy(data, offs)
    Bt = torch.from_numpy(B).cuda()
    for w in (_narrowest(M, lengths), 0.05, 0.6, 1.0):
        if any(math.floor(w * M * n) < max(M, n) for n in lengths):
            continue
        o = wts.options(band=w)
        score, cost, plen = (t.cpu().numpy() for t in wts.anomaly_score(Bt, gb, o))
        s32, c32, L32 = oracle.score(B, data, offs, "f32", band=w)
        assert (cost == c32).all() and (plen == L32).all(), w
        c2, p2, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(Bt, gb, o))
        assert (c2 == c32).all() and (p2 == L32).all(), w
        for k, y in enumerate(cyc):
            r = oracle.dtw(B, y, "f32", band=w)
            assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), (w, k)
        Bn, cnt, cb, ck = wts.dba_iterate(Bt, gb, o)
        Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(B, data, offs, "f32", band=w)
        assert (Bn.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all(), w


def test_band_one_is_unbanded_and_checkpoint_identical(wts):
    b = synth.config_batch(1, scale=0.05, T=10)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    B = torch.from_numpy(synth.clean_prototype(b, 1300)).cuda()
    ref = [t.cpu().numpy() for t in wts.dtw_align(B, gb)]
    one = [t.cpu().numpy() for t in wts.dtw_align(B, gb, wts.options(band=1.0))]
    for a, c in zip(ref, one):
        assert (a == c).all()
    stored = [t.cpu().numpy() for t in wts.dtw_align(B, gb, wts.options(band=0.3))]
    ckpt = [t.cpu().numpy() for t in wts.dtw_align(B, gb, wts.options(band=0.3, dir_mode=1, ckpt_bands=1))]
    for a, c in zip(stored, ckpt):
        assert (a == c).all()
    k = 3
    r = oracle.dtw(synth.clean_prototype(b, 1300), b.cycle(k), "f32", band=0.3)
    assert (stored[2][k] == r["jlo"]).all() and stored[1][k] == r["plen"]


def test_band_full_size_sampled(wts):
    """The DBA workload's shape (d = 6, M = 25,000, cycles 20k-30k) with
    Table I's band 0.6: two pairs against the oracle, the autotuned launch."""
    b = synth.config_batch(1, T=2)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bh = synth.clean_prototype(b, synth.PROTO_LEN[1])
    o = wts.options(band=0.6)
    cost, plen, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(torch.from_numpy(Bh).cuda(), gb, o))
    for k in range(2):
        r = oracle.dtw(Bh, b.cycle(k), "f32", path=False, band=0.6)
        assert cost[k] == r["cost"] and plen[k] == r["plen"], k
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k


def test_band_first_column_on_a_chunk_boundary(wts):
    """A row band whose first column is a multiple of 32 (M = N = 1100,
    w = 0.0295: row 512 starts at column 480, row 511 at 479) with a cycle that
    is the prototype shifted by 32 samples, so the optimal path runs along the
    band's left edge through (511, 479) -> (512, 480): the band's first cell
    takes its diagonal from the row above one column before the band starts."""
    M = N = 1100
    w = 0.0295
    assert math.ceil((512 * N - math.floor(w * M * N)) / M) == 480
    for seed in (5, 6):
        rng = np.random.default_rng(seed)
        B = rng.normal(size=(M, 2)).astype(np.float32)
        y = np.concatenate([B[32:], rng.normal(size=(32, 2)).astype(np.float32)])
        data, offs = _pack([y])
        gb = wts.Batch.from_numpy(data, offs)
        cost, plen, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(torch.from_numpy(B).cuda(), gb,
                                                                         wts.options(band=w)))
        r = oracle.dtw(B, y, "f32", band=w)
        assert r["jlo"][512] == 480 and r["jhi"][511] == 479
        assert cost[0] == r["cost"] and plen[0] == r["plen"]
        assert (jlo[0] == r["jlo"]).all() and (jhi[0] == r["jhi"]).all()

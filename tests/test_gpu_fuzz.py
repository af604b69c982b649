"""Seeded random configurations of the hard-min path against the oracle's
FP32 mirror, through the C ABI: channel count, prototype and cycle lengths
(across band, chunk and 2048-row segment edges), rows per lane, local cost,
Sakoe-Chiba band, stored or checkpointed codes.  Costs, |pi|, scores, paths
and one DBA iteration must be bit-exact in every combination.
"""
import numpy as np
import pytest

import oracle
from paper_2404_12134_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wts():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12134_gb300 import api, build
    build.build()
    return api


def _config(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.choice([1, 2, 3, 5, 6, 9]))
    M = int(rng.choice([1, 2, 31, 33, 511, 513, 1000, 2047, 2049, 3000, 4097, 5000]))
    T = int(rng.integers(1, 5))
    lens = [int(rng.choice([1, 2, 32, 33, 700, 1500, 2100, 3100, 4500])) for _ in range(T)]
    cost_kind = int(rng.integers(0, 2))
    band = 0.0
    if rng.random() < 0.35 and M > 1:
        # a width above the narrowest accepted one for every pair
        need = max(max(M, n) / (M * n) for n in lens)
        band = float(min(1.0, need * rng.uniform(1.05, 4.0)))
    dir_mode = int(rng.random() < 0.3)
    ckpt = int(rng.choice([1, 2, 16])) if dir_mode else 0
    if band > 0 or cost_kind == 1:
        R = int(rng.choice([0, 16]))
    else:
        R = int(rng.choice([0, 8, 16] + ([32] if d <= 3 else [])))
    walk = rng.random() < 0.5          # smooth signals (long runs of equal moves) or noise
    def series(n):
        x = rng.normal(size=(n, d))
        return (np.cumsum(x, 0) * 0.05 if walk else x).astype(np.float32)
    return dict(d=d, M=M, lens=lens, cost_kind=cost_kind, band=band, dir_mode=dir_mode, ckpt=ckpt, R=R,
                B=series(M), cyc=[series(n) for n in lens])


@pytest.mark.parametrize("seed", range(64))
def test_random_configuration_bit_exact(wts, seed):
    c = _config(1000 + seed)
    b = synth.pack(c["cyc"])
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(c["B"]).cuda()
    o = wts.options(rows_per_thread=c["R"], dir_mode=c["dir_mode"], ckpt_bands=c["ckpt"], band=c["band"],
                    cost_kind=c["cost_kind"])
    kw = dict(band=c["band"], cost_kind=c["cost_kind"])
    score, cost, plen = (t.cpu().numpy() for t in wts.anomaly_score(Bt, gb, o))
    s32, c32, L32 = oracle.score(c["B"], b.data, b.offsets, "f32", **kw)
    assert (cost == c32).all() and (plen == L32).all() and (score == s32).all(), c
    c2, p2, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(Bt, gb, o))
    assert (c2 == c32).all() and (p2 == L32).all(), c
    for k, y in enumerate(c["cyc"]):
        r = oracle.dtw(c["B"], y, "f32", path=False, **kw)
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), (k, c)
    Bn, cnt, cb, ck = wts.dba_iterate(Bt, gb, o)
    Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(c["B"], b.data, b.offsets, "f32", **kw)
    assert (Bn.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all(), c
    assert (ck.cpu().numpy() == ck_o).all() and float(cb) == cb_o, c


def _soft_config(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.choice([1, 2, 3, 5, 8]))
    M = int(rng.choice([1, 2, 33, 255, 257, 700, 1300]))
    T = int(rng.integers(1, 4))
    lens = [int(rng.choice([1, 2, 31, 33, 400, 900, 1400])) for _ in range(T)]
    gamma = float(rng.choice([0.01, 0.1, 1.0, 10.0]))
    cost_kind = int(rng.integers(0, 2))
    band = 0.0
    if rng.random() < 0.35 and M > 1:
        need = max(max(M, n) / (M * n) for n in lens)
        band = float(min(1.0, need * rng.uniform(1.05, 4.0)))
    dir_mode = int(rng.random() < 0.3)
    ckpt = int(rng.choice([1, 2, 16])) if dir_mode else 0
    return dict(d=d, M=M, lens=lens, gamma=gamma, cost_kind=cost_kind, band=band, dir_mode=dir_mode, ckpt=ckpt,
                B=rng.normal(size=(M, d)).astype(np.float32),
                cyc=[rng.normal(size=(n, d)).astype(np.float32) for n in lens])


@pytest.mark.parametrize("seed", range(24))
def test_random_softdtw_configuration(wts, seed):
    """Soft-DTW value and Eq. 7 gradient in random configurations against the
    FP64 oracle: values within 1e-5 of max(|v|, 1) or twice a plain FP32
    evaluation's error; gradients (relative to the largest component) within
    twice a plain FP32 evaluation's error plus 1e-5 plus (M + N) 2^-24: the
    kernel's weights come from the approximate hardware exponential (and, for
    the l2 cost, a fast division), one more rounding-size error per step of
    the E recursion, which compounds along the M + N steps of a path."""
    c = _soft_config(2000 + seed)
    b = synth.pack(c["cyc"])
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(c["B"]).cuda()
    o = wts.options(dir_mode=c["dir_mode"], ckpt_bands=c["ckpt"], band=c["band"], cost_kind=c["cost_kind"])
    ws = wts.Workspace()
    g_ = c["gamma"]
    w32 = (1.0 / np.asarray(c["lens"])).astype(np.float32)
    v = wts.softdtw_forward(Bt, gb, g_, o, ws=ws).cpu().numpy().astype(np.float64)
    g = wts.softdtw_backward(Bt, gb, g_, torch.from_numpy(w32).cuda(), o, ws=ws).cpu().numpy().astype(np.float64)
    assert wts.read_status(ws.buf) == 0
    kw = dict(band=c["band"], cost_kind=c["cost_kind"])
    vo, _, go = oracle.softdtw_batch(c["B"], b.data, b.offsets, g_, weights=w32.astype(np.float64), **kw)
    v32, _, g32 = oracle.softdtw_batch(c["B"], b.data, b.offsets, g_, weights=w32, prec="f32", **kw)
    vbar = np.maximum(1e-5 * np.maximum(np.abs(vo), 1.0), 2.0 * np.abs(v32.astype(np.float64) - vo))
    assert np.all(np.abs(v - vo) <= vbar), (c["M"], c["lens"], g_, np.abs(v - vo).max())
    scale = max(np.abs(go).max(), 1e-30)
    steps = c["M"] + max(c["lens"])
    bar = 2.0 * np.abs(g32.astype(np.float64) - go).max() / scale + 1e-5 + steps * 2.0 ** -24
    assert np.abs(g - go).max() / scale <= bar, (c["M"], c["lens"], g_, np.abs(g - go).max() / scale, bar)

"""Sub-DTW and the sliding-window segmentation (Sec. 3.2) on the GPU against
the CPU oracle: costs, piece bounds, |pi| and per-row ranges bit-exact to the
FP32 mirror."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_12134_gb300 import synth
from test_oracle_pins import pieces_match_cycles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wts():
    from paper_2404_12134_gb300 import api
    return api


def _pack(cyc):
    offs = np.concatenate([[0], np.cumsum([len(c) for c in cyc])]).astype(np.int64)
    return np.ascontiguousarray(np.concatenate(cyc).astype(np.float32)), offs


def _check(wts, X, cyc, rows=0):
    data, offs = _pack(cyc)
    gb = wts.Batch.from_numpy(data, offs)
    opts = wts.options(rows_per_thread=rows)
    cost, a, b, plen, jlo, jhi = (t.cpu().numpy() for t in wts.subdtw_align(torch.from_numpy(X).cuda(), gb, opts))
    for k, y in enumerate(cyc):
        r = oracle.subdtw(X, y, "f32")
        assert cost[k] == r["cost"], k
        assert (a[k], b[k], plen[k]) == (r["a"], r["b"], r["plen"]), k
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k
        r64 = oracle.subdtw(X, y, "f64")
        assert abs(cost[k] - r64["cost"]) <= 1e-5 * max(1.0, r64["cost"]), k


@pytest.mark.parametrize("rows", [16, 8, 4])
@pytest.mark.parametrize("M,lengths,d", [
    (1, [1, 7, 300], 1),
    (37, [1, 2, 40, 95], 3),
    (513, [600, 1100, 1], 2),          # two bands of 512 (R = 16), the second one row high
    (1100, [2200, 1733, 900], 9),      # three or five bands, ragged; windows of 2M and less
])
def test_subdtw_bit_exact(wts, M, lengths, d, rows):
    rng = np.random.default_rng(200 + M)
    X = rng.normal(size=(M, d)).astype(np.float32)
    _check(wts, X, [rng.normal(size=(n, d)).astype(np.float32) for n in lengths], rows)


def test_subdtw_integer_ties(wts):
    """Integer samples: many equal costs, so the first cheapest end column and
    the tie order decide; every window of 1..40 columns against 1..19 rows."""
    rng = np.random.default_rng(210)
    for M in (1, 2, 5, 19):
        X = rng.integers(-2, 3, size=(M, 2)).astype(np.float32)
        for rows in (16, 8):
            _check(wts, X, [rng.integers(-2, 3, size=(n, 2)).astype(np.float32) for n in range(1, 41)], rows)


def test_subdtw_embedded_copy(wts):
    rng = np.random.default_rng(211)
    X = rng.normal(size=(700, 3)).astype(np.float32)
    y = np.concatenate([rng.normal(size=(333, 3)) + 20, X, rng.normal(size=(600, 3)) - 20]).astype(np.float32)
    data, offs = _pack([y])
    gb = wts.Batch.from_numpy(data, offs)
    cost, a, b, plen, jlo, jhi = wts.subdtw_align(torch.from_numpy(X).cuda(), gb)
    assert float(cost[0]) == 0.0 and (int(a[0]), int(b[0]), int(plen[0])) == (333, 1032, 700)


@pytest.mark.parametrize("d,seed,rows", [(3, 7, 16), (9, 8, 16), (9, 8, 8), (9, 8, 4), (1, 9, 4)])
def test_segment_matches_oracle(wts, d, seed, rows):
    X, Y, bounds = synth.segmentation_stream(6, 550, 650, d, 600, seed)
    alpha = int(0.15 * len(X))
    got = wts.segment(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), alpha, wts.options(rows_per_thread=rows))
    ref = oracle.segment(X, Y, alpha, "f32")
    assert [(a, b) for a, b, c in got] == [(a, b) for a, b, c in ref]
    assert [c for a, b, c in got] == [float(c) for a, b, c in ref]


def test_segment_full_size(wts):
    """The paper's segmentation setting: a 16,300-sample reference with 9
    channels and windows of 2M.  The first window against the oracle cell for
    cell; the whole stream of 8 cycles against the generator's bounds."""
    X, Y, bounds = synth.segmentation_stream(8, 15000, 18000, 9, 16630, 9)
    M = len(X)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    data, offs = _pack([Y[:2 * M]])
    cost, a, b, plen, jlo, jhi = (t.cpu().numpy() for t in wts.subdtw_align(Xt, wts.Batch.from_numpy(data, offs)))
    r = oracle.subdtw(X, Y[:2 * M], "f32")
    assert cost[0] == r["cost"] and (a[0], b[0], plen[0]) == (r["a"], r["b"], r["plen"])
    assert (jlo[0] == r["jlo"]).all() and (jhi[0] == r["jhi"]).all()
    segs = wts.segment(Xt, Yt, int(0.15 * M))
    assert segs[0][:2] == (r["a"], r["b"]) and segs[0][2] == float(r["cost"])
    pieces_match_cycles(segs, bounds, len(bounds) - 1)
    # the library's default alpha is Sec. 3.2's 0.15 M (rounded down)
    assert wts.segment(Xt, Yt) == segs


def test_subdtw_rejects_unsupported_options(wts):
    X = torch.zeros((10, 1), device="cuda")
    gb = wts.Batch.from_numpy(np.zeros((20, 1), np.float32), np.array([0, 20], np.int64))
    with pytest.raises(Exception):
        wts.subdtw_align(X, gb, wts.options(rows_per_thread=32))
    with pytest.raises(Exception):
        wts.subdtw_align(X, gb, wts.options(dir_mode=1))

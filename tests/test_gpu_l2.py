"""GPU parity of the l2-norm local cost (wts_options.cost_kind = 1: delta is
the Euclidean norm itself, Sec. 3.2's wording, instead of its square) against
the CPU oracle, through the C ABI.

Bar: as for the squared cost.  DTW costs, |pi|, scores, paths, counts, DBA
prototypes, Sub-DTW bounds and the segmentation bit-exact against the FP32
mirror (the kernels take the IEEE square root of the same fused sum); costs
within 1e-5 of FP64.  Soft-DTW values within 1e-5 of FP64 relative to
max(|v|, 1); gradients within twice the error of a plain FP32 evaluation plus
1e-5 (the kernel's 1/delta is a fast division, 2 ulp).
"""
import numpy as np
import pytest

import oracle
from paper_2404_12134_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

L2 = 1


@pytest.fixture(scope="module")
def wts():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12134_gb300 import api, build
    build.build()
    return api


def _pack(cyc):
    b = synth.pack(cyc)
    return b.data, b.offsets


def _cases():
    rng = np.random.default_rng(901)
    out = []
    lens = [1, 2, 31, 33, 500, 1100]
    for d in (1, 3, 6):
        for M in (1, 513, 1100):
            cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in lens]
            out.append((f"real-d{d}-M{M}", rng.normal(size=(M, d)).astype(np.float32), cyc))
    # d = 1 integers: |b - y| is an exact integer, ties everywhere
    cyc = [rng.integers(-2, 3, size=(n, 1)).astype(np.float32) for n in (40, 129, 300)]
    out.append(("int-d1", rng.integers(-2, 3, size=(150, 1)).astype(np.float32), cyc))
    # a zero-padded channel count (d = 5 runs in D = 6)
    cyc = [rng.normal(size=(n, 5)).astype(np.float32) for n in (64, 600)]
    out.append(("pad-d5", rng.normal(size=(700, 5)).astype(np.float32), cyc))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_l2_score_and_paths_bit_exact(wts, case):
    _, B, cyc = case
    data, offs = _pack(cyc)
    gb = wts.Batch.from_numpy(data, offs)
    Bt = torch.from_numpy(B).cuda()
    o = wts.options(cost_kind=L2)
    score, cost, plen = (t.cpu().numpy() for t in wts.anomaly_score(Bt, gb, o))
    s32, c32, L32 = oracle.score(B, data, offs, "f32", cost_kind=L2)
    assert (cost == c32).all() and (plen == L32).all() and (score == s32).all()
    s64, c64, _ = oracle.score(B, data, offs, "f64", cost_kind=L2)
    assert (np.abs(cost - c64) / np.maximum(np.abs(c64), 1e-30)).max() <= 1e-5
    c2, p2, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(Bt, gb, o))
    assert (c2 == c32).all() and (p2 == L32).all()
    for k, y in enumerate(cyc):
        r = oracle.dtw(B, y, "f32", path=False, cost_kind=L2)
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k
    # the squared cost gives other paths on real data: the option is live
    if case[0].startswith("real") and B.shape[0] > 1:
        c_sq = wts.anomaly_score(Bt, gb)[1].cpu().numpy()
        assert not np.array_equal(c_sq, cost)


def test_l2_checkpointed_codes_identical(wts):
    rng = np.random.default_rng(902)
    B = rng.normal(size=(1300, 3)).astype(np.float32)
    cyc = [rng.normal(size=(n, 3)).astype(np.float32) for n in (1200, 700, 1500)]
    gb = wts.Batch.from_numpy(*_pack(cyc))
    Bt = torch.from_numpy(B).cuda()
    ref = [t.cpu().numpy() for t in wts.dtw_align(Bt, gb, wts.options(cost_kind=L2))]
    ck = [t.cpu().numpy() for t in wts.dtw_align(Bt, gb, wts.options(cost_kind=L2, dir_mode=1, ckpt_bands=1))]
    for a, b in zip(ref, ck):
        assert (a == b).all()


def test_l2_dba_iterations_bit_exact(wts):
    rng = np.random.default_rng(903)
    d = 3
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in (500, 640, 777, 512, 900)]
    data, offs = _pack(cyc)
    gb = wts.Batch.from_numpy(data, offs)
    B = cyc[0].copy()
    Bt = torch.from_numpy(B).cuda()
    o = wts.options(cost_kind=L2)
    for _ in range(3):
        Bn, cnt, cb, ck = wts.dba_iterate(Bt, gb, o)
        Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(B, data, offs, "f32", cost_kind=L2)
        assert (Bn.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all()
        assert (ck.cpu().numpy() == ck_o).all() and float(cb) == cb_o
        B, Bt = Bo, Bn


@pytest.mark.parametrize("w", [0.1, 0.3])
def test_l2_banded_bit_exact(wts, w):
    rng = np.random.default_rng(904)
    d = 2
    M = 1100
    lens = [1000, 1300, 1250]
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in lens]
    data, offs = _pack(cyc)
    gb = wts.Batch.from_numpy(data, offs)
    B = rng.normal(size=(M, d)).astype(np.float32)
    Bt = torch.from_numpy(B).cuda()
    o = wts.options(cost_kind=L2, band=w)
    score, cost, plen = (t.cpu().numpy() for t in wts.anomaly_score(Bt, gb, o))
    s32, c32, L32 = oracle.score(B, data, offs, "f32", band=w, cost_kind=L2)
    assert (cost == c32).all() and (plen == L32).all() and (score == s32).all()
    c2, p2, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(Bt, gb, o))
    for k, y in enumerate(cyc):
        r = oracle.dtw(B, y, "f32", path=False, band=w, cost_kind=L2)
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k


@pytest.mark.parametrize("M,lengths,d", [(37, [1, 40, 95], 3), (513, [600, 1100, 1], 2), (1100, [2200, 900], 9)])
def test_l2_subdtw_bit_exact(wts, M, lengths, d):
    rng = np.random.default_rng(905 + M)
    X = rng.normal(size=(M, d)).astype(np.float32)
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in lengths]
    gb = wts.Batch.from_numpy(*_pack(cyc))
    cost, a, b, plen, jlo, jhi = (t.cpu().numpy() for t in
                                  wts.subdtw_align(torch.from_numpy(X).cuda(), gb, wts.options(cost_kind=L2)))
    for k, y in enumerate(cyc):
        r = oracle.subdtw(X, y, "f32", cost_kind=L2)
        assert cost[k] == r["cost"] and (a[k], b[k], plen[k]) == (r["a"], r["b"], r["plen"]), k
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k


def test_l2_segment_matches_oracle(wts):
    X, Y, bounds = synth.segmentation_stream(6, 550, 650, 3, 600, 17)
    alpha = int(0.15 * len(X))
    got = wts.segment(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), alpha, wts.options(cost_kind=L2))
    ref = oracle.segment(X, Y, alpha, "f32", cost_kind=L2)
    assert [(a, b) for a, b, c in got] == [(a, b) for a, b, c in ref]
    assert [c for a, b, c in got] == [float(c) for a, b, c in ref]


def test_l2_pairwise_and_medoid(wts):
    rng = np.random.default_rng(906)
    cyc = [rng.normal(size=(n, 2)).astype(np.float32) for n in (90, 120, 75, 140, 100)]
    data, offs = _pack(cyc)
    C = wts.pairwise_dtw(wts.Batch.from_numpy(data, offs), wts.options(cost_kind=L2)).cpu().numpy()
    idx, Co = oracle.medoid(data, offs, cost_kind=L2)
    assert (C == Co).all()
    assert int(wts.medoid(torch.from_numpy(C).cuda())[0]) == idx


VALUE_TOL = 1e-5


@pytest.mark.parametrize("band", [0.0, 0.6])
@pytest.mark.parametrize("gamma", [1.0, 0.1])
@pytest.mark.parametrize("case", [(1, 64, [64, 40, 100], 1), (4, 513, [400, 600], 3), (5, 260, [650, 80], 6)],
                         ids=["M64-d1", "M513-d3", "M260-d6"])
def test_l2_softdtw_value_and_gradient(wts, case, gamma, band):
    seed, M, lens, d = case
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(M, d)).astype(np.float32)
    b = synth.pack([rng.normal(size=(n, d)).astype(np.float32) for n in lens])
    if band > 0 and any(np.floor(band * M * n) < max(M, n) for n in lens):
        pytest.skip("band narrower than max(M, N) for a pair")
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    o = wts.options(cost_kind=L2, band=band)
    ws = wts.Workspace()
    v = wts.softdtw_forward(Bt, gb, gamma, o, ws=ws)
    wts_w = (1.0 / np.asarray(lens)).astype(np.float32)
    g = wts.softdtw_backward(Bt, gb, gamma, torch.from_numpy(wts_w).cuda(), o, ws=ws)
    assert wts.read_status(ws.buf) == 0
    w64 = wts_w.astype(np.float64)
    vo, _, go = oracle.softdtw_batch(B, b.data, b.offsets, gamma, weights=w64, band=band, cost_kind=L2)
    vg = v.cpu().numpy().astype(np.float64)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(vg - vo) <= VALUE_TOL * np.maximum(np.abs(vo), 1.0)), np.abs(vg - vo).max()
    g32 = oracle.softdtw_batch(B, b.data, b.offsets, gamma, weights=wts_w, prec="f32", band=band, cost_kind=L2)[2]
    bar = 2.0 * np.abs(g32.astype(np.float64) - go).max() / np.abs(go).max() + 1e-5
    err = np.abs(gg - go).max() / np.abs(go).max()
    assert err <= bar, (err, bar)


def test_l2_softdtw_zero_distance(wts):
    """B equal to the cycle: the diagonal distances are 0, where the norm has
    no derivative; the gradient takes 0 there and stays finite, as the
    oracle's."""
    rng = np.random.default_rng(907)
    X = rng.normal(size=(300, 2)).astype(np.float32)
    b = synth.pack([X.copy(), rng.normal(size=(250, 2)).astype(np.float32)])
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(X).cuda()
    o = wts.options(cost_kind=L2)
    ws = wts.Workspace()
    wts.softdtw_forward(Bt, gb, 0.5, o, ws=ws)
    w = np.array([1.0 / 300, 1.0 / 250], dtype=np.float32)
    g = wts.softdtw_backward(Bt, gb, 0.5, torch.from_numpy(w).cuda(), o, ws=ws).cpu().numpy().astype(np.float64)
    assert np.isfinite(g).all()
    _, _, go = oracle.softdtw_batch(X, b.data, b.offsets, 0.5, weights=w.astype(np.float64), cost_kind=L2)
    g32 = oracle.softdtw_batch(X, b.data, b.offsets, 0.5, weights=w, prec="f32", cost_kind=L2)[2]
    bar = 2.0 * np.abs(g32.astype(np.float64) - go).max() / np.abs(go).max() + 1e-5
    assert np.abs(g - go).max() / np.abs(go).max() <= bar


def test_l2_rejects_other_row_counts(wts):
    rng = np.random.default_rng(908)
    gb = wts.Batch.from_numpy(*_pack([rng.normal(size=(50, 2)).astype(np.float32)]))
    B = torch.from_numpy(rng.normal(size=(40, 2)).astype(np.float32)).cuda()
    for r in (8, 32):
        with pytest.raises(RuntimeError):
            wts.anomaly_score(B, gb, wts.options(cost_kind=L2, rows_per_thread=r))

"""GPU parity of the hard-min path (DTW, |pi|, score, alignment ranges, DBA)
against the CPU oracle, through the C ABI.

Bar: costs, |pi|, scores, paths, counts and DBA prototypes bit-exact against
the oracle's FP32 mirror (same tie rule, same float operation order); against
the FP64 oracle the relative error of costs / scores is stated and held to
1e-5.
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


def _gb(wts, data, offs):
    return wts.Batch.from_numpy(data, offs)


def _pack(cycles):
    b = synth.pack(cycles)
    return b.data, b.offsets


def _cases():
    rng = np.random.default_rng(101)
    out = []
    # ragged lengths around the 32-column chunk and the 512-row band edges
    lens = [1, 2, 31, 32, 33, 97, 500, 1100]
    for d in (1, 3, 6):
        for M in (1, 5, 511, 512, 513, 1100):
            cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in lens]
            B = rng.normal(size=(M, d)).astype(np.float32)
            out.append((f"real-d{d}-M{M}", B, cyc))
    # integer samples: frequent exact ties exercise the tie rule
    for d in (1, 2):
        cyc = [rng.integers(-2, 3, size=(n, d)).astype(np.float32) for n in (40, 77, 129, 300)]
        B = rng.integers(-2, 3, size=(150, d)).astype(np.float32)
        out.append((f"int-d{d}", B, cyc))
    # odd channel counts that run zero-padded (d=5 in D=6, d=9 in D=12)
    for d in (5, 9):
        cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in (64, 600)]
        out.append((f"pad-d{d}", rng.normal(size=(700, d)).astype(np.float32), cyc))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_anomaly_score_bit_exact(wts, case):
    _, B, cyc = case
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    score, cost, plen = wts.anomaly_score(torch.from_numpy(B).cuda(), gb)
    s32, c32, L32 = oracle.score(B, data, offs, "f32")
    assert (cost.cpu().numpy() == c32).all()
    assert (plen.cpu().numpy() == L32).all()
    assert (score.cpu().numpy() == s32).all()
    s64, c64, L64 = oracle.score(B, data, offs, "f64")
    rel = np.abs(cost.cpu().numpy() - c64) / np.maximum(np.abs(c64), 1e-30)
    assert rel.max() <= 1e-5, rel.max()


@pytest.mark.parametrize("case", CASES[::2], ids=[c[0] for c in CASES[::2]])
def test_dtw_align_paths_bit_exact(wts, case):
    _, B, cyc = case
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    cost, plen, jlo, jhi = wts.dtw_align(torch.from_numpy(B).cuda(), gb)
    cost, plen, jlo, jhi = (t.cpu().numpy() for t in (cost, plen, jlo, jhi))
    for k, y in enumerate(cyc):
        r = oracle.dtw(B, y, "f32")
        assert cost[k] == r["cost"], k
        assert plen[k] == r["plen"], k
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k


@pytest.mark.parametrize("rows,warps,order", [(8, 4, 0), (8, 1, 1), (16, 1, 0), (16, 3, 1), (32, 4, 0), (32, 2, 1)])
def test_launch_variants_agree(wts, rows, warps, order):
    rng = np.random.default_rng(102)
    cyc = [rng.normal(size=(n, 2)).astype(np.float32) for n in (3, 700, 1500, 1031)]
    B = rng.normal(size=(1300, 2)).astype(np.float32)
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    opts = wts.options(rows_per_thread=rows, warps_per_block=warps, keep_batch_order=order)
    Bt = torch.from_numpy(B).cuda()
    score, cost, plen = wts.anomaly_score(Bt, gb, opts)
    c2, p2, jlo, jhi = wts.dtw_align(Bt, gb, opts)
    s32, c32, L32 = oracle.score(B, data, offs, "f32")
    assert (cost.cpu().numpy() == c32).all() and (plen.cpu().numpy() == L32).all()
    assert (c2.cpu().numpy() == c32).all() and (p2.cpu().numpy() == L32).all()
    r = oracle.dtw(B, cyc[2], "f32")
    assert (jlo[2].cpu().numpy() == r["jlo"]).all() and (jhi[2].cpu().numpy() == r["jhi"]).all()


def test_dba_iterations_bit_exact(wts):
    """Ten DBA iterations from the medoid on the small DBA workload at full
    size (16 cycles of 1.0-1.2k): every iteration's prototype, counts and cost
    equal the FP32 mirror's."""
    b = synth.config_batch(0)
    gb = _gb(wts, b.data, b.offsets)
    C = wts.pairwise_dtw(gb)
    idx, sums = wts.medoid(C)
    k0, C_or = oracle.medoid(b.data, b.offsets)
    assert (C.cpu().numpy() == C_or).all()
    assert int(idx) == k0
    B = b.cycle(k0).copy()
    Bg = torch.from_numpy(B).cuda()
    for it in range(10):
        Bn, cnt, cb, ck = wts.dba_iterate(Bg, gb)
        Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(B, b.data, b.offsets, "f32")
        assert (Bn.cpu().numpy() == Bo).all(), it
        assert (cnt.cpu().numpy() == cnt_o).all(), it
        assert float(cb) == cb_o, it
        assert (ck.cpu().numpy() == ck_o).all(), it
        B, Bg = Bo, Bn
    assert wts.read_status(wts._default_ws[torch.cuda.current_device()].buf) == 0


def test_dba_fixed_point(wts):
    rng = np.random.default_rng(103)
    x = rng.normal(size=(777, 3)).astype(np.float32)
    data, offs = _pack([x, x, x, x])
    Bn, cnt, cb, ck = wts.dba_iterate(torch.from_numpy(x).cuda(), _gb(wts, data, offs))
    assert (Bn.cpu().numpy() == x).all() and float(cb) == 0.0 and (cnt.cpu().numpy() == 4).all()


def test_init_helpers_bit_exact(wts):
    b = synth.config_batch(2, scale=0.05)
    gb = _gb(wts, b.data, b.offsets)
    for M in (1, 7, 500, 1001):
        got = wts.euclid_mean(gb, M).cpu().numpy()
        assert (got == oracle.euclid_mean(b.data, b.offsets, M)).all(), M
        x = b.cycle(3)
        got = wts.resample(torch.from_numpy(x).cuda(), M).cpu().numpy()
        assert (got == oracle.resample(x, M)).all(), M


def test_full_size_sampled_pair(wts):
    """Full workload-1 shape (d = 6, M = 25,000, cycles 20k-30k) in the same
    launch configuration as the benchmark: one pair checked cell-for-cell on
    its path against the oracle, the others by path properties."""
    b = synth.config_batch(1, T=3)
    gb = _gb(wts, b.data, b.offsets)
    B = synth.clean_prototype(b, synth.PROTO_LEN[1])
    cost, plen, jlo, jhi = wts.dtw_align(torch.from_numpy(B).cuda(), gb)
    cost, plen, jlo, jhi = (t.cpu().numpy() for t in (cost, plen, jlo, jhi))
    r = oracle.dtw(B, b.cycle(1), "f32", path=False)
    assert cost[1] == r["cost"] and plen[1] == r["plen"]
    assert (jlo[1] == r["jlo"]).all() and (jhi[1] == r["jhi"]).all()
    for k in range(3):
        N = b.lengths[k]
        assert jlo[k, 0] == 0 and jhi[k, -1] == N - 1
        assert ((jlo[k, 1:] == jhi[k, :-1]) | (jlo[k, 1:] == jhi[k, :-1] + 1)).all()
        assert int((jhi[k] - jlo[k] + 1).sum()) == plen[k]
    s, c, L = wts.anomaly_score(torch.from_numpy(B).cuda(), gb)
    assert (c.cpu().numpy() == cost).all() and (L.cpu().numpy() == plen).all()


@pytest.mark.parametrize("G,rows", [(1, 16), (2, 16), (3, 16), (16, 16), (3, 8), (5, 8)])
def test_checkpoint_recompute_paths_identical(wts, G, rows):
    """dir_mode=1 keeps only the band hand-off rows and recomputes G bands of
    codes at a time during the backtrack: same paths, costs and |pi|."""
    rng = np.random.default_rng(104)
    cyc = [rng.normal(size=(n, 3)).astype(np.float32) for n in (5, 800, 1777, 2100)]
    B = rng.normal(size=(2600, 3)).astype(np.float32)          # 6 bands of 512 rows, ragged last band
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    Bt = torch.from_numpy(B).cuda()
    ref = [t.cpu().numpy() for t in wts.dtw_align(Bt, gb, wts.options(rows_per_thread=rows))]
    got = [t.cpu().numpy() for t in wts.dtw_align(Bt, gb, wts.options(rows_per_thread=rows, dir_mode=1, ckpt_bands=G))]
    for a, b in zip(ref, got):
        assert (a == b).all()
    r = oracle.dtw(B, cyc[3], "f32")
    assert (got[2][3] == r["jlo"]).all() and (got[3][3] == r["jhi"]).all() and got[1][3] == r["plen"]


def test_checkpoint_dba_identical(wts):
    b = synth.config_batch(1, scale=0.05, T=12)
    gb = _gb(wts, b.data, b.offsets)
    B = synth.clean_prototype(b, 1300)
    Bs = torch.from_numpy(B).cuda()
    Bc = Bs.clone()
    opt = wts.options(dir_mode=1, ckpt_bands=2)
    for it in range(3):
        Bs2, cs, cbs, _ = wts.dba_iterate(Bs, gb)
        Bc2, cc, cbc, _ = wts.dba_iterate(Bc, gb, opt)
        assert torch.equal(Bs2, Bc2) and torch.equal(cs, cc) and float(cbs) == float(cbc), it
        Bs, Bc = Bs2, Bc2


def test_edge_shapes(wts):
    """Single-row and single-column pairs, 16 channels (the maximum), and many
    tiny cycles in one launch (the work list orders thousands of pairs)."""
    rng = np.random.default_rng(105)
    cases = []
    cases.append((rng.normal(size=(1, 4)).astype(np.float32), [rng.normal(size=(n, 4)).astype(np.float32) for n in (1, 5, 300)]))
    cases.append((rng.normal(size=(900, 2)).astype(np.float32), [rng.normal(size=(1, 2)).astype(np.float32)] * 3))
    cases.append((rng.normal(size=(530, 16)).astype(np.float32), [rng.normal(size=(n, 16)).astype(np.float32) for n in (7, 640)]))
    cases.append((rng.normal(size=(40, 1)).astype(np.float32),
                  [rng.normal(size=(int(n), 1)).astype(np.float32) for n in rng.integers(1, 6, size=3000)]))
    for B, cyc in cases:
        data, offs = _pack(cyc)
        gb = _gb(wts, data, offs)
        Bt = torch.from_numpy(B).cuda()
        score, cost, plen = wts.anomaly_score(Bt, gb)
        s32, c32, L32 = oracle.score(B, data, offs, "f32")
        assert (cost.cpu().numpy() == c32).all() and (plen.cpu().numpy() == L32).all()
        c2, p2, jlo, jhi = wts.dtw_align(Bt, gb)
        for k in (0, len(cyc) - 1):
            r = oracle.dtw(B, cyc[k], "f32")
            assert (jlo[k].cpu().numpy() == r["jlo"]).all() and (jhi[k].cpu().numpy() == r["jhi"]).all()


def test_full_size_uneven_scoring_sampled(wts):
    """The full uneven-scoring workload (1,000 cycles, 3 channels, lengths
    2k-60k, M = 20,000) in the benchmark's launch shape (autotuned, one
    graph-captured launch): the longest cycle and two others checked against
    the oracle; every |pi| within [max(M, N), M + N - 1]."""
    b = synth.config_batch(3)
    gb = _gb(wts, b.data, b.offsets)
    B = synth.clean_prototype(b, synth.PROTO_LEN[3])
    Bt = torch.from_numpy(B).cuda()
    opts, _ = wts.autotune(wts._abi.OP_ANOMALY_SCORE, Bt, gb)
    ws = wts.Workspace()
    g, (score, cost, plen) = wts.capture(lambda: wts.anomaly_score(Bt, gb, opts, ws=ws))
    g.replay()
    cost, plen = cost.cpu().numpy(), plen.cpu().numpy()
    N = b.lengths
    M = B.shape[0]
    assert ((plen >= np.maximum(M, N)) & (plen <= M + N - 1)).all()
    for k in (int(np.argmax(N)), 0, 517):
        r = oracle.dtw(B, b.cycle(k), "f32", path=False)
        assert cost[k] == r["cost"] and plen[k] == r["plen"], k


@pytest.mark.parametrize("d", [1, 6, 16])
def test_half_word_codes(wts, d):
    """Eight rows per lane: two steps' codes share one word, so an even and an
    odd number of steps (N + 31) both close their last word; several bands of
    256 rows with a ragged last band."""
    rng = np.random.default_rng(106 + d)
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in (1, 2, 257, 600, 601, 1023)]
    B = rng.normal(size=(1100, d)).astype(np.float32)
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    Bt = torch.from_numpy(B).cuda()
    o8 = wts.options(rows_per_thread=8)
    cost, plen, jlo, jhi = (t.cpu().numpy() for t in wts.dtw_align(Bt, gb, o8))
    score, c2, p2 = wts.anomaly_score(Bt, gb, o8)
    s32, c32, L32 = oracle.score(B, data, offs, "f32")
    assert (cost == c32).all() and (plen == L32).all()
    assert (c2.cpu().numpy() == c32).all() and (p2.cpu().numpy() == L32).all()
    for k, y in enumerate(cyc):
        r = oracle.dtw(B, y, "f32")
        assert (jlo[k] == r["jlo"]).all() and (jhi[k] == r["jhi"]).all(), k
    Bn, cnt, cb, ck = wts.dba_iterate(Bt, gb, o8)
    Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(B, data, offs, "f32")
    assert (Bn.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all()


def test_segmented_walk_any_guess(wts):
    """Prototype rows cut into three 2048-row segments, walked at once: the
    paths are the oracle's whatever the range arrays hold on entry (the walk
    reads them as guesses): all columns 0, invalid values, the right answer,
    a wrong path; and DBA iterations reusing their workspace."""
    rng = np.random.default_rng(77)
    d = 3
    M = 5000
    walk = lambda n: np.cumsum(rng.normal(size=(n, d)), 0).astype(np.float32) * 0.1
    B = walk(M)
    cyc = [walk(n) for n in (4000, 5200, 6100, 1, 2047)]
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    Bt = torch.from_numpy(B).cuda()
    ref = [oracle.dtw(B, y, "f32", path=False) for y in cyc]
    T = len(cyc)
    ws = wts.Workspace()

    def check(jlo, jhi):
        c, pl, lo, hi = wts.dtw_align(Bt, gb, ws=ws, jlo=jlo, jhi=jhi)
        c, pl, lo, hi = (t.cpu().numpy() for t in (c, pl, lo, hi))
        for k, r in enumerate(ref):
            assert c[k] == r["cost"] and pl[k] == r["plen"], k
            assert (lo[k] == r["jlo"]).all() and (hi[k] == r["jhi"]).all(), k
        return lo, hi

    z = torch.zeros((T, M), dtype=torch.int32, device="cuda")
    check(z.clone(), z.clone())
    check(torch.full((T, M), -7, dtype=torch.int32, device="cuda"), torch.full((T, M), 1 << 30, dtype=torch.int32,
                                                                            device="cuda"))
    lo, hi = check(None, None)
    good_lo, good_hi = torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda()
    check(good_lo.clone(), good_hi.clone())
    # another pair's path as the guess
    check(good_lo.roll(1, 0).contiguous(), good_hi.roll(1, 0).contiguous())
    # DBA iterations on one workspace: each walk guesses from the previous one
    wsd = wts.Workspace()
    Bc = B.copy()
    for _ in range(2):
        Bn, cnt, cb, ck = wts.dba_iterate(torch.from_numpy(Bc).cuda(), gb, ws=wsd)
        Bo, cnt_o, cb_o, _ = oracle.dba_iterate(Bc, data, offs, "f32")
        assert (Bn.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all() and float(cb) == cb_o
        Bc = Bo


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_score_via_codes_bit_exact(wts, case):
    """anomaly_score through stored codes and the walk (score_via_codes = 1)
    gives the FP32 mirror's cost, |pi| and score, bit for bit, as the count
    inside the DP does."""
    _, B, cyc = case
    data, offs = _pack(cyc)
    gb = _gb(wts, data, offs)
    ws = wts.Workspace()
    score, cost, plen = wts.anomaly_score(torch.from_numpy(B).cuda(), gb, wts.options(score_via_codes=1), ws=ws)
    assert wts.read_status(ws.buf) == 0
    s32, c32, L32 = oracle.score(B, data, offs, "f32")
    assert (cost.cpu().numpy() == c32).all()
    assert (plen.cpu().numpy() == L32).all()
    assert (score.cpu().numpy() == s32).all()


@pytest.mark.parametrize("rows,dir_mode", [(16, 0), (32, 0), (8, 0), (16, 1)])
def test_score_via_codes_long_prototype(wts, rows, dir_mode):
    """Several 2,048-row segments of the walk (M = 5,000) and checkpointed
    codes: the codes form equals the count inside the DP and the FP32 mirror."""
    b = synth.config_batch(3, scale=0.25, T=6)
    B = synth.clean_prototype(b, 5000)
    gb = _gb(wts, b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    ref = wts.anomaly_score(Bt, gb, ws=ws)
    got = wts.anomaly_score(Bt, gb, wts.options(rows_per_thread=rows, dir_mode=dir_mode, ckpt_bands=3,
                                                 score_via_codes=1), ws=ws)
    assert wts.read_status(ws.buf) == 0
    for x, y in zip(got, ref):
        assert torch.equal(x, y)
    s32, c32, L32 = oracle.score(B, b.data, b.offsets, "f32")
    assert (got[2].cpu().numpy() == L32).all() and (got[1].cpu().numpy() == c32).all()


def test_autotune_score_forms(wts):
    """With a workspace that holds the codes, the score's autotuner also times
    the codes form; whatever it picks gives the same scores."""
    from paper_2404_12134_gb300 import _abi
    b = synth.config_batch(3, scale=0.2, T=12)
    B = synth.clean_prototype(b, 4000)
    gb = _gb(wts, b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    best, ms = wts.autotune(_abi.OP_ANOMALY_SCORE, Bt, gb, ws)
    assert ms > 0 and best.score_via_codes in (0, 1)
    got = wts.anomaly_score(Bt, gb, best, ws=ws)
    ref = wts.anomaly_score(Bt, gb, ws=ws)
    for x, y in zip(got, ref):
        assert torch.equal(x, y)

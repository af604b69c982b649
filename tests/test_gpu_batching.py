"""Batching and scheduling (one persistent launch over uneven pairs, the
autotuner, CUDA-graph capture): results stay bit-exact against the oracle's
FP32 mirror whatever launch shape is chosen or replayed."""
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


def _uneven(seed=31, T=40, d=3):
    b = synth.config_batch(3, scale=0.02, T=T)      # log-normal lengths, 3 channels, anomalies
    M = 400
    B = synth.clean_prototype(b, M)
    return b, B


def test_autotuned_options_are_exact(wts):
    b, B = _uneven()
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    for op in (wts._abi.OP_ANOMALY_SCORE, wts._abi.OP_DTW_ALIGN):
        opts, ms = wts.autotune(op, Bt, gb)
        assert opts.rows_per_thread in (8, 16, 32) and 1 <= opts.warps_per_block <= 4 and ms > 0
        again, _ = wts.autotune(op, Bt, gb)          # cached
        assert (again.rows_per_thread, again.warps_per_block) == (opts.rows_per_thread, opts.warps_per_block)
    s, c, L = wts.anomaly_score(Bt, gb, opts)
    s32, c32, L32 = oracle.score(B, b.data, b.offsets, "f32")
    assert (c.cpu().numpy() == c32).all() and (L.cpu().numpy() == L32).all() and (s.cpu().numpy() == s32).all()


def test_graph_replay_follows_inputs(wts):
    b, B = _uneven(T=24)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    g, (score, cost, plen) = wts.capture(lambda: wts.anomaly_score(Bt, gb, ws=ws))
    g.replay()
    s32, c32, L32 = oracle.score(B, b.data, b.offsets, "f32")
    assert (cost.cpu().numpy() == c32).all() and (plen.cpu().numpy() == L32).all()
    # new prototype values in the same buffer: the replay recomputes
    B2 = (B * 0.5 + 0.25).astype(np.float32)
    Bt.copy_(torch.from_numpy(B2))
    g.replay()
    s32, c32, L32 = oracle.score(B2, b.data, b.offsets, "f32")
    assert (cost.cpu().numpy() == c32).all() and (plen.cpu().numpy() == L32).all()
    assert (score.cpu().numpy() == s32).all()


def test_dba_iteration_in_a_graph(wts):
    b = synth.config_batch(0, scale=0.2)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    B0 = b.cycle(0).copy()
    Bin = torch.from_numpy(B0).cuda()
    ws = wts.Workspace()
    g, (Bout, cnt, cb, ck) = wts.capture(lambda: wts.dba_iterate(Bin, gb, ws=ws))
    Bo = B0
    for it in range(3):
        g.replay()
        Bo, cnt_o, cb_o, _ = oracle.dba_iterate(Bo, b.data, b.offsets, "f32")
        assert (Bout.cpu().numpy() == Bo).all() and float(cb) == cb_o, it
        Bin.copy_(Bout)


def test_one_launch_per_pair_matches_batched(wts):
    b, B = _uneven(T=12)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    s, c, L = wts.anomaly_score(Bt, gb)
    for k in range(b.T):
        o0, o1 = int(b.offsets[k]), int(b.offsets[k + 1])
        one = wts.Batch(gb.data[o0:o1], torch.tensor([0, o1 - o0], device="cuda"), np.array([0, o1 - o0]))
        sk, ck, Lk = wts.anomaly_score(Bt, one)
        assert float(ck[0]) == float(c[k]) and int(Lk[0]) == int(L[k])


def test_segmented_dba_iteration_in_a_graph(wts):
    """A prototype of three 2048-row segments: the segmented walk's rounds and
    its last kernel are captured with the rest of the iteration; each replay
    guesses from the paths the previous replay left in the workspace."""
    rng = np.random.default_rng(55)
    walk = lambda n: (np.cumsum(rng.normal(size=(n, 2)), 0) * 0.05).astype(np.float32)
    cyc = [walk(n) for n in (4100, 4700, 3900)]
    b = synth.pack(cyc)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    B0 = walk(4500)
    Bin = torch.from_numpy(B0).cuda()
    ws = wts.Workspace()
    g, (Bout, cnt, cb, ck) = wts.capture(lambda: wts.dba_iterate(Bin, gb, ws=ws))
    Bo = B0
    for it in range(3):
        g.replay()
        Bo, cnt_o, cb_o, _ = oracle.dba_iterate(Bo, b.data, b.offsets, "f32")
        assert (Bout.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all() and float(cb) == cb_o, it
        Bin.copy_(Bout)


@pytest.mark.parametrize("wpb,max_blocks,rows", [(1, 1, 8), (1, 2, 16), (4, 3, 8), (2, 5, 16), (4, 0, 32)])
def test_grouped_work_list_any_group_size(wts, wpb, max_blocks, rows):
    """The work list takes the pairs in groups of about (resident warps /
    bands per pair), band-major within a group: with a grid cut to a few
    warps the groups have 1 to a few pairs and the last group is ragged (one
    warp alone runs every item in turn).  Scores, costs, |pi|, paths and the
    DBA prototype stay bit-exact against the FP32 mirror."""
    b, B = _uneven(seed=33, T=13)
    M = 700                                  # 3 bands of 256 rows, 2 of 512 or 1 of 1,024
    B = synth.clean_prototype(b, M)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    opt = wts.options(rows_per_thread=rows, warps_per_block=wpb, max_blocks=max_blocks)
    s, c, L = wts.anomaly_score(Bt, gb, opt)
    s32, c32, L32 = oracle.score(B, b.data, b.offsets, "f32")
    assert (c.cpu().numpy() == c32).all() and (L.cpu().numpy() == L32).all() and (s.cpu().numpy() == s32).all()
    Bn, cnt, cb, ck = wts.dba_iterate(Bt, gb, opt)
    Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(B, b.data, b.offsets, "f32")
    assert (Bn.cpu().numpy() == Bo).all() and (cnt.cpu().numpy() == cnt_o).all() and (ck.cpu().numpy() == ck_o).all()

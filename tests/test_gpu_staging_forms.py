"""GPU parity of the paper's data forms through the C ABI: last-value padding
(Sec. 4.1) and one joint's channel (Sec. 5), bit-exact against the oracle's
definitions; the per-joint scores and the padded Soft-DTW that the paper
computes, against the oracle on the same forms."""
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


def _batch(rng, lens, d):
    return synth.pack([rng.normal(size=(n, d)).astype(np.float32) for n in lens])


@pytest.mark.parametrize("lens,d,L", [([5, 9, 1, 7], 3, 0), ([1], 1, 0), ([300, 1000, 999, 2], 6, 1500),
                                      ([40000, 3], 2, 0)])
def test_pad_last_bit_exact(wts, lens, d, L):
    b = _batch(np.random.default_rng(len(lens) + d), lens, d)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    pb = wts.pad_last(gb, L)
    want = oracle.pad_last(b.data, b.offsets, L)
    assert pb.T == len(lens) and pb.d == d
    assert (pb.data.cpu().numpy().reshape(want.shape) == want).all()
    assert (pb.offsets.cpu().numpy() == np.arange(len(lens) + 1) * want.shape[1]).all()


def test_pad_last_rejects_short_length(wts):
    b = _batch(np.random.default_rng(3), [10, 20], 2)
    with pytest.raises(RuntimeError):
        wts.pad_last(wts.Batch.from_numpy(b.data, b.offsets), 19)


def test_select_channel_bit_exact(wts):
    b = _batch(np.random.default_rng(4), [100, 3000, 1, 57], 5)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    for c in range(5):
        one = wts.select_channel(gb, c)
        assert one.d == 1 and one.T == 4
        assert (one.data.cpu().numpy()[:, 0] == oracle.select_channel(b.data, c)).all()
    with pytest.raises(RuntimeError):
        wts.select_channel(gb, 5)


def test_per_joint_scores(wts):
    """The paper scores each joint against its own barycenter: d = 1 scores
    on the selected channels, bit-exact against the oracle on the slices."""
    rng = np.random.default_rng(5)
    b = _batch(rng, [700, 1100, 520], 3)
    B = rng.normal(size=(600, 3)).astype(np.float32)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    for c in range(3):
        one = wts.select_channel(gb, c)
        Bc = np.ascontiguousarray(B[:, c:c + 1])
        score, cost, plen = (t.cpu().numpy() for t in wts.anomaly_score(torch.from_numpy(Bc).cuda(), one))
        s32, c32, L32 = oracle.score(Bc, oracle.select_channel(b.data, c), b.offsets, "f32")
        assert (cost == c32).all() and (plen == L32).all() and (score == s32).all()


def test_padded_softdtw_as_in_the_paper(wts):
    """Soft-DTW on the last-value padded batch (the paper's setting for its
    Soft-DTW runs) against the oracle on the padded arrays."""
    rng = np.random.default_rng(6)
    b = _batch(rng, [300, 410, 380], 1)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    pb = wts.pad_last(gb)
    P = oracle.pad_last(b.data, b.offsets)
    B = rng.normal(size=(350, 1)).astype(np.float32)
    v = wts.softdtw_forward(torch.from_numpy(B).cuda(), pb, 1.0).cpu().numpy().astype(np.float64)
    for k in range(3):
        # the value (about -1.5) is a small difference of path sums in the
        # hundreds: the bar is twice a plain FP32 evaluation's error plus 1e-5
        vo = oracle.softdtw(B, P[k], 1.0, "f64", want_grad=False)["value"]
        v32 = float(oracle.softdtw(B, P[k], 1.0, "f32", want_grad=False)["value"])
        assert abs(v[k] - vo) <= 2.0 * abs(v32 - vo) + 1e-5 * max(1.0, abs(vo)), (k, v[k], vo, v32)

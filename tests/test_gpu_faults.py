"""Failure detection without a GPU fault: every in-kernel wait is bounded.

A host-set option makes the band producers skip their hand-off rows (a slot
that nothing ever fills); the consumers' waits give up after a short poll
limit, raise the workspace status and abort word, and every warp leaves.  The
call itself returns normally (it is asynchronous); the status read afterwards
is WTS_ETIMEOUT, and the next normal call on the same workspace is correct.
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


def _case():
    rng = np.random.default_rng(51)
    B = rng.normal(size=(1300, 2)).astype(np.float32)         # several bands: consumers exist
    cyc = [rng.normal(size=(n, 2)).astype(np.float32) for n in (700, 900)]
    b = synth.pack(cyc)
    return B, b


@pytest.mark.parametrize("call", ["score", "align", "soft"])
def test_wait_gives_up_and_reports(wts, call):
    from paper_2404_12134_gb300._abi import WTS_ETIMEOUT
    B, b = _case()
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    bad = wts.options(fault_skip_handoff=1, spin_limit=2000)
    if call == "score":
        wts.anomaly_score(Bt, gb, bad, ws=ws)
    elif call == "align":
        wts.dtw_align(Bt, gb, bad, ws=ws)
    else:
        wts.softdtw_forward(Bt, gb, 0.5, bad, ws=ws)
    assert wts.read_status(ws.buf) == WTS_ETIMEOUT
    # the context is intact: a normal call on the same workspace is exact
    s, c, L = wts.anomaly_score(Bt, gb, ws=ws)
    assert wts.read_status(ws.buf) == 0
    s32, c32, L32 = oracle.score(B, b.data, b.offsets, "f32")
    assert (c.cpu().numpy() == c32).all() and (L.cpu().numpy() == L32).all()


def _nonfinite_case(where, value):
    B, b = _case()
    B = B.copy()
    data = b.data.copy()
    if where == "cycle":
        data[int(b.offsets[1]) + 37, 1] = value       # one sample of the second cycle
    else:
        B[611, 0] = value                             # one prototype sample
    return B, synth.pack([data[int(b.offsets[k]):int(b.offsets[k + 1])] for k in range(b.T)])


CALL_WHERE = [(c, w) for c in ("score", "align", "dba", "soft", "subdtw") for w in ("cycle", "prototype")] + \
    [("pairwise", "cycle")]                                   # the pairwise matrix has no prototype


@pytest.mark.parametrize("value", [np.nan, np.inf, -np.inf], ids=["nan", "inf", "-inf"])
@pytest.mark.parametrize("call,where", CALL_WHERE)
def test_nonfinite_sample_is_rejected_on_the_device(wts, call, where, value):
    """Sec. 3.1 removes missing values before alignment: a NaN or +-inf sample
    is found by the device-side scan before any DP work, every kernel of the
    call leaves at once, and the workspace status reads WTS_EINVAL (not a
    timeout: a short poll limit makes a regression show as WTS_ETIMEOUT
    quickly).  The next call on the same workspace is exact."""
    from paper_2404_12134_gb300._abi import WTS_EINVAL
    B, b = _nonfinite_case(where, value)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    o = wts.options(spin_limit=1 << 16)
    if call == "score":
        wts.anomaly_score(Bt, gb, o, ws=ws)
    elif call == "align":
        wts.dtw_align(Bt, gb, o, ws=ws)
    elif call == "dba":
        wts.dba_iterate(Bt, gb, o, ws=ws)
    elif call == "soft":
        wts.softdtw_forward(Bt, gb, 0.5, o, ws=ws)
        wts.softdtw_backward(Bt, gb, 0.5, None, o, ws=ws)
    elif call == "subdtw":
        wts.subdtw_align(Bt, gb, o, ws=ws)
    else:
        wts.pairwise_dtw(gb, o, ws=ws)
    assert wts.read_status(ws.buf) == WTS_EINVAL
    B0, b0 = _case()
    gb0 = wts.Batch.from_numpy(b0.data, b0.offsets)
    s, c, L = wts.anomaly_score(torch.from_numpy(B0).cuda(), gb0, ws=ws)
    assert wts.read_status(ws.buf) == 0
    s32, c32, L32 = oracle.score(B0, b0.data, b0.offsets, "f32")
    assert (c.cpu().numpy() == c32).all() and (L.cpu().numpy() == L32).all()


def test_softdtw_overflowing_finite_samples_never_look_unwritten(wts):
    """Finite samples whose squared differences overflow FP32 make the soft
    recursion produce NaN; the kernels store such a value in a hand-off slot
    as -inf, so a consumer never mistakes it for a slot still unwritten: the
    forward and backward finish without a timeout."""
    B, b = _case()
    big = (b.data * np.float32(3e19)).astype(np.float32)
    bb = synth.pack([big[int(b.offsets[k]):int(b.offsets[k + 1])] for k in range(b.T)])
    assert np.isfinite(bb.data).all()
    gb = wts.Batch.from_numpy(bb.data, bb.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    o = wts.options(spin_limit=1 << 20)
    wts.softdtw_forward(Bt, gb, 0.5, o, ws=ws)
    wts.softdtw_backward(Bt, gb, 0.5, None, o, ws=ws)
    assert wts.read_status(ws.buf) == 0

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

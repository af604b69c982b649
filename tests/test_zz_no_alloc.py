"""anomaly_score_noalloc: the scoring entry point for callers that cannot
allocate device memory (a host that owns and budgets all device memory, or a
scoring loop that must not stall on cudaMalloc / cudaFree).  It must give the
same output as anomaly_score, call after call, although every call reuses the
library's one fixed scratch array.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_12134_gb300 import _abi, build, synth

torch = pytest.importorskip("torch")


def _lib():
    build.build()
    return _abi.load()


@pytest.mark.gpu
def test_noalloc_matches_anomaly_score_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12134_gb300 import api
    _lib()
    rng = np.random.default_rng(4242)
    calls = [
        (rng.normal(size=(700, 3)), [rng.normal(size=(n, 3)) for n in (1, 650, 1033)]),
        (rng.normal(size=(1100, 1)), [rng.normal(size=(n, 1)) for n in (2047, 31)]),
    ]
    got = []
    for B, cyc in calls:
        b = synth.pack([c.astype(np.float32) for c in cyc])
        gb = api.Batch.from_numpy(b.data, b.offsets)
        Bt = torch.from_numpy(B.astype(np.float32)).cuda()
        got.append((api.anomaly_score_noalloc(Bt, gb), Bt, gb))
    for (na, Bt, gb) in got:
        ref = api.anomaly_score(Bt, gb)
        for x, y in zip(na, ref):
            assert torch.equal(x, y)


@pytest.mark.gpu
def test_noalloc_status_is_readable():
    """The fixed scratch's device status word is readable by the caller: a
    wait made to give up (host-set fault injection, short poll limit) shows as
    WTS_ETIMEOUT, a non-finite sample as WTS_EINVAL, and the next normal call
    reads WTS_OK with the same output as anomaly_score."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12134_gb300 import api
    _lib()
    rng = np.random.default_rng(99)
    B = rng.normal(size=(1300, 2)).astype(np.float32)          # several bands: hand-off waits exist
    cyc = [rng.normal(size=(n, 2)).astype(np.float32) for n in (700, 900)]
    b = synth.pack(cyc)
    gb = api.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    api.anomaly_score_noalloc(Bt, gb, api.options(fault_skip_handoff=1, spin_limit=2000))
    assert api.noalloc_status() == _abi.WTS_ETIMEOUT
    bad = b.data.copy()
    bad[5, 1] = np.nan
    gbad = api.Batch.from_numpy(bad, b.offsets)
    api.anomaly_score_noalloc(Bt, gbad, api.options(spin_limit=1 << 16))
    assert api.noalloc_status() == _abi.WTS_EINVAL
    got = api.anomaly_score_noalloc(Bt, gb)
    assert api.noalloc_status() == _abi.WTS_OK
    ref = api.anomaly_score(Bt, gb)
    for x, y in zip(got, ref):
        assert torch.equal(x, y)


def test_noalloc_rejects_oversized_batch_before_launch():
    lib = _lib()
    lengths = np.array([30000] * 8, dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    b = _abi.wts_batch()
    b.data = 256
    b.offsets = 256
    b.offsets_host = offs.ctypes.data
    b.T = 8
    b.d = 6
    rc = lib.anomaly_score_noalloc(256, 25000, ctypes.byref(b), None, None, 256, None, None)
    assert rc == _abi.WTS_ENOMEM
    assert b"fixed scratch" in lib.wts_last_error()

"""Batch staging (Sec. 3.1): time steps with a missing value are removed on
the GPU exactly as the plain definition removes them, and the compacted batch
aligns exactly as the oracle aligns the same series."""
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


def _raw(T=9, d=3, seed=61):
    rng = np.random.default_rng(seed)
    base = synth.BaseSignal(rng, d, "bumps")
    cyc = [synth.make_cycle(rng, base, int(n), gaps="nan") for n in rng.integers(300, 3000, size=T)]
    cyc[2][5, 1] = np.nan                     # one missing channel drops the whole step
    cyc[4][:] = np.nan                        # a cycle with nothing left
    return cyc


def test_compaction_matches_definition(wts):
    cyc = _raw()
    raw = synth.pack(cyc)
    gb = wts.Batch.from_numpy(raw.data, raw.offsets)
    out = wts.compact_nan(gb)
    kept = [c[~np.isnan(c).any(axis=1)] for c in cyc]
    lens = np.array([len(c) for c in kept])
    assert (np.diff(out.offsets_host) == lens).all() and lens[4] == 0
    assert (out.data.cpu().numpy() == np.concatenate(kept)).all()


def test_compacted_batch_scores_like_oracle(wts):
    cyc = [c for i, c in enumerate(_raw(seed=62)) if i != 4]
    raw = synth.pack(cyc)
    out = wts.compact_nan(wts.Batch.from_numpy(raw.data, raw.offsets))
    kept = synth.pack([c[~np.isnan(c).any(axis=1)] for c in cyc])
    B = kept.cycle(0)[:700].copy()
    s, c, L = wts.anomaly_score(torch.from_numpy(B).cuda(), out)
    s32, c32, L32 = oracle.score(B, kept.data, kept.offsets, "f32")
    assert (c.cpu().numpy() == c32).all() and (L.cpu().numpy() == L32).all()


def test_compaction_at_scale(wts):
    """Full batched-DBA size: 200 cycles x 6 ch with 2 % missing steps."""
    rng = np.random.default_rng(63)
    base = synth.BaseSignal(rng, 6, "bumps")
    lens = rng.integers(20000, 30001, size=200)
    cyc = [synth.make_cycle(rng, base, int(n), gaps="nan") for n in lens]
    raw = synth.pack(cyc)
    out = wts.compact_nan(wts.Batch.from_numpy(raw.data, raw.offsets))
    keep = ~np.isnan(raw.data).any(axis=1)
    assert out.offsets_host[-1] == keep.sum()
    assert (out.data.cpu().numpy() == raw.data[keep]).all()

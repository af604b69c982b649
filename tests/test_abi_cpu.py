"""The C-ABI library loads and exports every symbol include/wetsand.h declares.

No compute call is made (no GPU here); only host-side sizing and argument
validation, which the library does before touching CUDA.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2404_12134_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "wetsand.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?!typedef\b)(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"anomaly_score", "dtw_align", "dba_iterate"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(_abi.EXPORTS) == names


def test_version(lib):
    assert lib.wts_version() >= 100


def _batch(lengths, d=1):
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    b = _abi.wts_batch()
    b.data = 16          # never dereferenced by host-only calls
    b.offsets = 16
    b.offsets_host = offs.ctypes.data
    b.T = len(lengths)
    b.d = d
    return b, offs


def _size(lib, op, M, b, opts=None):
    n = ctypes.c_size_t(0)
    rc = lib.wts_workspace_size(op, M, ctypes.byref(b), ctypes.byref(opts) if opts else None, ctypes.byref(n))
    return rc, n.value


def test_workspace_sizes(lib):
    b, offs = _batch([1000, 1200, 37], d=6)
    rc, score = _size(lib, _abi.OP_ANOMALY_SCORE, 1100, b)
    assert rc == 0 and score > 0
    rc, align = _size(lib, _abi.OP_DTW_ALIGN, 1100, b)
    assert rc == 0
    # 2-bit codes: about M*N/4 bytes per cycle plus the skew margin
    cells = 1100 * (1000 + 1200 + 37)
    assert cells / 4 <= align - score <= cells / 4 * 2.5
    rc, dba = _size(lib, _abi.OP_DBA_ITERATE, 1100, b)
    assert rc == 0 and dba > align
    # eight rows per lane: two steps' codes per word, the same 2 bits per cell
    o = _abi.wts_options()
    o.rows_per_thread = 8
    rc, score8 = _size(lib, _abi.OP_ANOMALY_SCORE, 1100, b, o)
    rc2, align8 = _size(lib, _abi.OP_DTW_ALIGN, 1100, b, o)
    assert rc == 0 and rc2 == 0
    assert cells / 4 <= align8 - score8 <= cells / 4 * 2.5


def test_validation_errors(lib):
    b, offs = _batch([10, 0, 5])
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 8, b)[0] == _abi.WTS_EINVAL
    assert b"length" in lib.wts_last_error()
    b, offs = _batch([10, 5], d=17)
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 8, b)[0] == _abi.WTS_EINVAL
    b, offs = _batch([10, 5])
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 0, b)[0] == _abi.WTS_EINVAL
    assert _size(lib, 99, 8, b)[0] == _abi.WTS_EINVAL
    o = _abi.wts_options()
    o.rows_per_thread = 24
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 8, b, o)[0] == _abi.WTS_EINVAL
    b6, _ = _batch([10, 5], d=6)
    o.rows_per_thread = 32
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 8, b6, o)[0] == _abi.WTS_EINVAL
    bp, _ = _batch([10])
    assert _size(lib, _abi.OP_PAIRWISE, 0, bp)[0] == _abi.WTS_EINVAL
    # a too-small workspace is rejected before any launch
    b, offs = _batch([10, 5])
    rc = lib.anomaly_score(256, 8, ctypes.byref(b), None, 256, 16, None, 256, None, None)
    assert rc == _abi.WTS_ENOMEM
    rc = lib.dba_iterate(256, 256, 8, ctypes.byref(b), None, 256, 1 << 30, None, None, None, None)
    assert rc == _abi.WTS_EINVAL and b"alias" in lib.wts_last_error()


def test_checkpoint_mode_shrinks_workspace(lib):
    b, offs = _batch([110000] * 4, d=3)
    o = _abi.wts_options()
    rc, stored = _size(lib, _abi.OP_DBA_ITERATE, 110000, b)
    o.dir_mode = 1
    o.ckpt_bands = 16
    rc2, ckpt = _size(lib, _abi.OP_DBA_ITERATE, 110000, b, o)
    assert rc == 0 and rc2 == 0
    # codes: M*N/4 bytes per cycle stored, vs 16 bands of 512 rows recomputed at a time
    assert stored > 4 * 110000 * 110000 / 4
    assert ckpt < stored / 8
    o.dir_mode = 2
    assert _size(lib, _abi.OP_DBA_ITERATE, 110000, b, o)[0] == _abi.WTS_EINVAL


def test_subdtw_workspace_and_validation(lib):
    b, offs = _batch([1200, 37], d=9)
    rc, sub = _size(lib, _abi.OP_SUBDTW, 600, b)
    rc2, align = _size(lib, _abi.OP_DTW_ALIGN, 600, b)
    # the same codes; dtw_align adds the segmented walk's state (16 bytes per
    # pair and segment of 2048 rows, in a 256-byte aligned block)
    assert rc == 0 and rc2 == 0 and sub + 256 >= align
    o = _abi.wts_options()
    o.rows_per_thread = 8
    assert _size(lib, _abi.OP_SUBDTW, 600, b, o)[0] == 0
    o.rows_per_thread = 32
    assert _size(lib, _abi.OP_SUBDTW, 600, b, o)[0] == _abi.WTS_EINVAL
    # four rows per lane: Sub-DTW windows only
    o.rows_per_thread = 4
    assert _size(lib, _abi.OP_SUBDTW, 600, b, o)[0] == 0
    for op in (_abi.OP_ANOMALY_SCORE, _abi.OP_DTW_ALIGN, _abi.OP_DBA_ITERATE, _abi.OP_PAIRWISE):
        assert _size(lib, op, 600, b, o)[0] == _abi.WTS_EINVAL
        assert b"Sub-DTW only" in lib.wts_last_error()
    o.rows_per_thread = 0
    o.dir_mode = 1
    assert _size(lib, _abi.OP_SUBDTW, 600, b, o)[0] == _abi.WTS_EINVAL
    n = ctypes.c_size_t(0)
    assert lib.wts_segment_workspace_size(16300, 9, None, ctypes.byref(n)) == 0
    # two window slots of 2M columns: about 2 * M * 2M / 4 bytes of codes
    assert 2 * 16300 * 32600 / 4 <= n.value <= 2 * 16300 * 32600 / 4 * 1.2
    assert lib.wts_segment_workspace_size(0, 9, None, ctypes.byref(n)) == _abi.WTS_EINVAL


def test_band_option_layout_and_validation(lib):
    """wts_options keeps its 64-byte layout with the double band field; a band
    narrower than max(M, N) for some pair, a band with 8 rows per lane, and a
    band on a non-DTW operation are refused on the host."""
    assert ctypes.sizeof(_abi.wts_options) == 64
    assert _abi.wts_options.band.offset == 32
    b, offs = _batch([1200, 800], d=3)
    o = _abi.wts_options()
    o.band = 0.6
    for op in (_abi.OP_ANOMALY_SCORE, _abi.OP_DTW_ALIGN, _abi.OP_DBA_ITERATE):
        assert _size(lib, op, 1000, b, o)[0] == 0
    o.band = 1199 / (1000 * 1200)             # floor(w M N) < max(M, N) for the first pair
    assert _size(lib, _abi.OP_DTW_ALIGN, 1000, b, o)[0] == _abi.WTS_EINVAL
    assert b"too narrow" in lib.wts_last_error()
    o.band = 0.6
    o.rows_per_thread = 8
    assert _size(lib, _abi.OP_DTW_ALIGN, 1000, b, o)[0] == _abi.WTS_EINVAL
    o.rows_per_thread = 0
    assert _size(lib, _abi.OP_SOFTDTW, 1000, b, o)[0] == 0
    assert _size(lib, _abi.OP_SUBDTW, 1000, b, o)[0] == _abi.WTS_EINVAL
    o.band = -1.0
    assert _size(lib, _abi.OP_DTW_ALIGN, 1000, b, o)[0] == _abi.WTS_EINVAL


def test_cost_kind_option_layout_and_validation(lib):
    """cost_kind sits after the band in the same 64 bytes; 0 and 1 are the only
    values; the l2-norm DTW kernels hold 16 rows per lane (8 or 32 refused, 0
    means 16, also where d <= 2 would otherwise pick 32); soft-DTW takes it
    with its own row count; the segmentation workspace follows R = 16."""
    assert ctypes.sizeof(_abi.wts_options) == 64
    assert _abi.wts_options.cost_kind.offset == 40
    b, offs = _batch([1200, 800], d=2)
    o = _abi.wts_options()
    o.cost_kind = 1
    for op in (_abi.OP_ANOMALY_SCORE, _abi.OP_DTW_ALIGN, _abi.OP_DBA_ITERATE, _abi.OP_SOFTDTW, _abi.OP_SUBDTW,
               _abi.OP_PAIRWISE):
        assert _size(lib, op, 1000, b, o)[0] == 0, op
    # default R for d = 2 is 32 (two bands of 1024 rows); with the l2 norm, 16
    # (two of 512): the code store of dtw_align is the same size, the hand-off
    # rows are not
    o0 = _abi.wts_options()
    o16 = _abi.wts_options()
    o16.rows_per_thread = 16
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 1000, b, o)[1] == _size(lib, _abi.OP_ANOMALY_SCORE, 1000, b, o16)[1]
    assert _size(lib, _abi.OP_ANOMALY_SCORE, 1000, b, o)[1] != _size(lib, _abi.OP_ANOMALY_SCORE, 1000, b, o0)[1]
    for r in (8, 32):
        o.rows_per_thread = r
        assert _size(lib, _abi.OP_DTW_ALIGN, 1000, b, o)[0] == _abi.WTS_EINVAL
        assert b"l2-norm" in lib.wts_last_error()
    o.rows_per_thread = 0
    o.band = 0.6
    assert _size(lib, _abi.OP_DTW_ALIGN, 1000, b, o)[0] == 0
    assert _size(lib, _abi.OP_SOFTDTW, 1000, b, o)[0] == 0
    o.band = 0.0
    for bad in (2, -1):
        o.cost_kind = bad
        assert _size(lib, _abi.OP_ANOMALY_SCORE, 1000, b, o)[0] == _abi.WTS_EINVAL
        assert b"cost_kind" in lib.wts_last_error()
    o.cost_kind = 1
    n16 = ctypes.c_size_t(0)
    n8 = ctypes.c_size_t(0)
    assert lib.wts_segment_workspace_size(600, 3, ctypes.byref(o), ctypes.byref(n16)) == 0
    assert lib.wts_segment_workspace_size(600, 3, None, ctypes.byref(n8)) == 0
    o16.cost_kind = 0
    n16b = ctypes.c_size_t(0)
    assert lib.wts_segment_workspace_size(600, 3, ctypes.byref(o16), ctypes.byref(n16b)) == 0
    assert n16.value == n16b.value


def test_score_via_codes_workspace(lib):
    """The score through stored codes needs the code store of dtw_align plus
    the walk's ranges; the count inside the DP needs neither."""
    b, offs = _batch([3000, 2500, 777], d=3)
    o = _abi.wts_options()
    o.score_via_codes = 1
    rc, via = _size(lib, _abi.OP_ANOMALY_SCORE, 2600, b, o)
    rc2, fused = _size(lib, _abi.OP_ANOMALY_SCORE, 2600, b)
    rc3, align = _size(lib, _abi.OP_DTW_ALIGN, 2600, b)
    assert rc == rc2 == rc3 == 0
    assert via > align > fused
    o.score_via_codes = 2
    rc, _ = _size(lib, _abi.OP_ANOMALY_SCORE, 2600, b, o)
    assert rc == _abi.WTS_EINVAL


def test_softdtw_checkpoint_workspace(lib):
    """Soft-DTW checkpoint mode without a band keeps column checkpoints (R/14
    of the stored R's size), with a band two groups of R."""
    b, offs = _batch([9000, 11000], d=1)
    rc, stored = _size(lib, _abi.OP_SOFTDTW, 10000, b)
    o = _abi.wts_options()
    o.dir_mode = 1
    rc2, ck = _size(lib, _abi.OP_SOFTDTW, 10000, b, o)
    o.band = 0.6
    o.ckpt_bands = 4
    rc3, banded = _size(lib, _abi.OP_SOFTDTW, 10000, b, o)
    assert rc == rc2 == rc3 == 0
    cells = 10000 * 20000
    assert stored >= 4 * cells and ck < stored / 10 and ck > 4 * cells * 9 / (8 * 16) * 0.9
    assert banded < stored / 4


def test_softdtw_store_pairs_workspace(lib):
    """store_pairs (column checkpoints, no band): the first pairs of the
    longest-first order keep R; the workspace grows by exactly their R minus
    their checkpoints, from dir_mode = 1's size (none kept) to dir_mode = 0's
    (all kept); any other use is rejected."""
    lengths = [9000, 11000, 5000]
    M = 10000
    b, offs = _batch(lengths, d=1)
    rc, stored = _size(lib, _abi.OP_SOFTDTW, M, b)
    o = _abi.wts_options()
    o.dir_mode = 1
    rc1, ck = _size(lib, _abi.OP_SOFTDTW, M, b, o)
    assert rc == rc1 == 0
    nb = -(-M // 256)                                  # bands of 32 lanes x 8 rows

    def extra(n):                                      # floats: R minus column checkpoints of one pair
        return nb * (n + 31) * 32 * 8 - nb * (-(-(n + 31) // 16)) * 9 * 32

    want = {0: 0, 1: extra(11000), 2: extra(11000) + extra(9000), 3: sum(extra(n) for n in lengths)}
    for S, dx in want.items():
        o.store_pairs = S
        rc, sz = _size(lib, _abi.OP_SOFTDTW, M, b, o)
        assert rc == 0
        assert abs(sz - ck - 4 * dx) < 256, (S, sz - ck, 4 * dx)
    assert sz == stored
    o.store_pairs = 7                                  # more than T: every pair
    assert _size(lib, _abi.OP_SOFTDTW, M, b, o) == (0, stored)
    # in batch order (keep_batch_order) the first pairs of the batch keep R
    o.store_pairs = 1
    o.keep_batch_order = 1
    rc, sz = _size(lib, _abi.OP_SOFTDTW, M, b, o)
    assert rc == 0 and abs(sz - ck - 4 * extra(9000)) < 256
    o.keep_batch_order = 0
    # the Adam and L-BFGS drivers take the same option
    assert _size(lib, _abi.OP_SOFTDTW_ADAM, M, b, o)[0] == 0
    o.store_pairs = -1
    assert _size(lib, _abi.OP_SOFTDTW, M, b, o)[0] == _abi.WTS_EINVAL
    o.store_pairs = 1
    o.dir_mode = 0
    assert _size(lib, _abi.OP_SOFTDTW, M, b, o)[0] == _abi.WTS_EINVAL
    o.dir_mode = 1
    o.band = 0.6
    assert _size(lib, _abi.OP_SOFTDTW, M, b, o)[0] == _abi.WTS_EINVAL
    o.band = 0.0
    assert _size(lib, _abi.OP_DTW_ALIGN, M, b, o)[0] == _abi.WTS_EINVAL
    assert b"store_pairs" in lib.wts_last_error()


def test_store_pairs_for_memory(lib):
    """api.store_pairs_for_memory sizes soft-DTW's store_pairs by the free
    device memory: the most pairs whose workspace (the library's own size)
    fits in free memory less the margin."""
    from paper_2404_12134_gb300 import api
    lengths = [9000, 11000, 5000, 10000]
    M = 10000
    _, offs = _batch(lengths, d=3)

    class FakeBatch:                                   # host-only sizing: no device data is touched
        T = len(lengths)

        def c(self):
            b = _abi.wts_batch()
            b.data = 16
            b.offsets = 16
            b.offsets_host = offs.ctypes.data
            b.T = self.T
            b.d = 3
            return b

    sizes = [api.workspace_size(_abi.OP_SOFTDTW, M, FakeBatch(), api.options(dir_mode=1, store_pairs=s))
             for s in range(5)]
    assert sizes == sorted(sizes) and sizes[0] < sizes[1]
    margin = 16 * 10**9
    for free, want in ((sizes[0] + 1, 0), (sizes[2] + margin, 2), (sizes[2] + margin - 1, 1),
                       (sizes[4] + margin + 10**9, 4)):
        got, need = api.store_pairs_for_memory(M, FakeBatch(), free_bytes=free, margin_bytes=margin,
                                               opts=api.options(cost_kind=1, dir_mode=0))
        assert got == want, (free, got, want)
        want_need = api.workspace_size(_abi.OP_SOFTDTW, M, FakeBatch(),
                                       api.options(cost_kind=1, dir_mode=1, store_pairs=want)) if want else 0
        assert need == want_need


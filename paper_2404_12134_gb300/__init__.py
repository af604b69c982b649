"""GB300-native (sm_103a) alignment hot path of WETSAND (arXiv 2404.12134).

The compute lives in ``libwetsand.so`` (hand-written CUDA behind the C ABI of
``include/wetsand.h``); ``api`` is the thin Python binding.  Importing this
package does not touch CUDA; the first call loads the library and fails loudly
if it is missing (there is no CPU fallback).  ``synth`` is the seeded input
generator.
"""
from __future__ import annotations

_API_NAMES = {
    "Batch", "Workspace", "options", "workspace_size", "read_status", "anomaly_score", "dtw_align",
    "dba_iterate", "pairwise_dtw", "medoid", "resample", "euclid_mean", "profile_enable", "profile_read",
    "anomaly_score_noalloc", "softdtw_forward", "softdtw_backward", "adam_step", "SoftDTW", "softdtw",
    "softdtw_barycenter", "autotune", "capture", "peak_probe", "compact_nan",
}


def __getattr__(name):
    if name in _API_NAMES:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)

"""Python binding of the C ABI (argument marshalling only).

Every function takes CUDA tensors, builds the C structs, hands raw device
pointers and the current torch stream to ``libwetsand.so`` and returns the
output tensors.  No step of the method runs here; PyTorch supplies device
memory (outputs and the workspace, from its caching allocator) and the stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from ._abi import check, wts_batch, wts_options


class Batch:
    """A packed batch of T cycles resident on the GPU (Sec. 3.1 layout).

    data [sum N_k, d] float32 (CUDA), offsets [T+1] int64 (CUDA) plus the host
    copy of the offsets, which the library uses to plan the work."""

    def __init__(self, data: torch.Tensor, offsets: torch.Tensor, offsets_host: np.ndarray | None = None):
        if data.dim() == 1:
            data = data[:, None]
        if not (data.is_cuda and data.dtype == torch.float32 and data.is_contiguous()):
            raise ValueError("data must be a contiguous float32 CUDA tensor")
        if not (offsets.is_cuda and offsets.dtype == torch.int64 and offsets.is_contiguous()):
            raise ValueError("offsets must be a contiguous int64 CUDA tensor")
        self.data = data
        self.offsets = offsets
        if offsets_host is None:
            offsets_host = offsets.cpu().numpy()
        self.offsets_host = np.ascontiguousarray(offsets_host, dtype=np.int64)
        self.T = int(self.offsets_host.shape[0] - 1)
        self.d = int(data.shape[1])

    @classmethod
    def from_numpy(cls, data: np.ndarray, offsets: np.ndarray, device="cuda") -> "Batch":
        d = torch.from_numpy(np.ascontiguousarray(data, dtype=np.float32)).to(device)
        o = torch.from_numpy(np.ascontiguousarray(offsets, dtype=np.int64)).to(device)
        return cls(d, o, offsets)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets_host)

    def c(self) -> wts_batch:
        b = wts_batch()
        b.data = self.data.data_ptr()
        b.offsets = self.offsets.data_ptr()
        b.offsets_host = self.offsets_host.ctypes.data
        b.T = self.T
        b.d = self.d
        return b


def options(rows_per_thread=0, warps_per_block=0, max_blocks=0, keep_batch_order=0, dir_mode=0,
            ckpt_bands=0, spin_limit=0, fault_skip_handoff=0, band=0.0, cost_kind=0,
            score_via_codes=0, store_pairs=0) -> wts_options:
    """Launch and method options (see wts_options in include/wetsand.h); band > 0
    is the Sakoe-Chiba width (Table I) for the DTW operations; cost_kind 1 takes
    the l2 norm as the local cost instead of its square (Sec. 3.2);
    score_via_codes 1 makes anomaly_score walk stored codes for |pi|;
    store_pairs keeps R of the longest pairs in soft-DTW's checkpoint mode."""
    o = wts_options()
    o.store_pairs = store_pairs
    o.score_via_codes = score_via_codes
    o.band = float(band)
    o.cost_kind = cost_kind
    o.rows_per_thread = rows_per_thread
    o.warps_per_block = warps_per_block
    o.max_blocks = max_blocks
    o.keep_batch_order = keep_batch_order
    o.dir_mode = dir_mode
    o.ckpt_bands = ckpt_bands
    o.spin_limit = spin_limit
    o.fault_skip_handoff = fault_skip_handoff
    return o


def _opt(opts):
    return ctypes.byref(opts) if opts is not None else None


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _p(t: torch.Tensor | None):
    return None if t is None else t.data_ptr()


class Workspace:
    """A reusable device buffer from torch's allocator, grown on demand."""

    def __init__(self, device=None):
        self.device = torch.device("cuda" if device is None else device)
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf

    def status(self) -> int:
        return read_status(self.buf)


_default_ws: dict = {}


def release_default_workspaces():
    """Drop the per-device workspaces that calls without an explicit
    Workspace share (their memory returns to torch's allocator)."""
    _default_ws.clear()


def _ws(ws: Workspace | None, nbytes: int) -> torch.Tensor:
    if ws is None:
        dev = torch.cuda.current_device()
        ws = _default_ws.setdefault(dev, Workspace(dev))
    return ws.get(nbytes)


def workspace_size(op: int, M: int, batch: Batch, opts=None) -> int:
    n = ctypes.c_size_t(0)
    check(_abi.load().wts_workspace_size(op, M, ctypes.byref(batch.c()), _opt(opts), ctypes.byref(n)))
    return n.value


def store_pairs_for_memory(M: int, batch: Batch, free_bytes: int | None = None, margin_bytes: int = 16 * 10**9,
                           opts=None) -> tuple[int, int]:
    """For soft-DTW's checkpoint mode (dir_mode = 1, no band): the most
    pairs that can keep R (wts_options.store_pairs) with the workspace
    within free_bytes (default: the current device's free memory) less
    margin_bytes.  Returns (store_pairs, workspace bytes); (0, 0) if even one
    stored pair does not fit.  opts supplies the other options (its dir_mode
    and store_pairs are overridden)."""
    if free_bytes is None:
        torch.cuda.empty_cache()
        free_bytes = torch.cuda.mem_get_info()[0]
    o = wts_options()
    if opts is not None:
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opts), ctypes.sizeof(o))
    o.dir_mode = 1
    best, need = 0, 0
    for s in range(1, batch.T + 1):
        o.store_pairs = s
        n = workspace_size(_abi.OP_SOFTDTW, M, batch, o)
        if n > free_bytes - margin_bytes:
            break
        best, need = s, n
    return best, need


def read_status(buf: torch.Tensor) -> int:
    s = ctypes.c_int32(0)
    check(_abi.load().wts_read_status(buf.data_ptr(), _stream(), ctypes.byref(s)))
    return s.value


def profile_enable(enable: bool = True):
    """Record CUDA events around every stage of the library's calls (measurement)."""
    check(_abi.load().wts_profile_enable(1 if enable else 0))


def profile_read(kernel: str = ""):
    """(total ms, kernel launches) of the recorded runs of one stage ("" = all);
    a stage may launch several kernels (the segmented backtrack's rounds)."""
    ms = ctypes.c_double(0)
    n = ctypes.c_int32(0)
    check(_abi.load().wts_profile_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def peak_probe(which: int) -> float:
    """Measured lane-ops/s: 0 FP32 FMA, 1 FP32 min/max, 2 MUFU ex2, 3 MUFU lg2,
    4 packed f32x2 FMA (2 lane-ops each), 5 three-input min."""
    v = ctypes.c_double(0)
    check(_abi.load().wts_peak_probe(which, ctypes.byref(v)))
    return v.value


def _check_B(B: torch.Tensor, d: int) -> torch.Tensor:
    if B.dim() == 1:
        B = B[:, None]
    if not (B.is_cuda and B.dtype == torch.float32 and B.is_contiguous()) or B.shape[1] != d:
        raise ValueError(f"prototype must be a contiguous float32 CUDA tensor [M, {d}]")
    return B


def anomaly_score(B: torch.Tensor, batch: Batch, opts=None, ws: Workspace | None = None):
    """Eq. 8 per cycle: (score [T], cost [T], plen [T])."""
    B = _check_B(B, batch.d)
    M = B.shape[0]
    lib = _abi.load()
    nb = workspace_size(_abi.OP_ANOMALY_SCORE, M, batch, opts)
    buf = _ws(ws, nb)
    dev = B.device
    score = torch.empty(batch.T, dtype=torch.float32, device=dev)
    cost = torch.empty(batch.T, dtype=torch.float32, device=dev)
    plen = torch.empty(batch.T, dtype=torch.int32, device=dev)
    check(lib.anomaly_score(B.data_ptr(), M, ctypes.byref(batch.c()), _opt(opts), buf.data_ptr(), buf.numel(),
                            _stream(), score.data_ptr(), cost.data_ptr(), plen.data_ptr()))
    return score, cost, plen


def anomaly_score_noalloc(B: torch.Tensor, batch: Batch, opts=None):
    """anomaly_score for callers that cannot allocate device memory: the
    library's fixed 32 MiB scratch replaces the workspace (small batches only;
    calls must not overlap on the GPU).  Outputs are allocated here by torch
    only for convenience; a C caller passes its own.  The scratch's device
    status is read by noalloc_status()."""
    B = _check_B(B, batch.d)
    M = B.shape[0]
    dev = B.device
    score = torch.empty(batch.T, dtype=torch.float32, device=dev)
    cost = torch.empty(batch.T, dtype=torch.float32, device=dev)
    plen = torch.empty(batch.T, dtype=torch.int32, device=dev)
    check(_abi.load().anomaly_score_noalloc(B.data_ptr(), M, ctypes.byref(batch.c()), _opt(opts), _stream(),
                                            score.data_ptr(), cost.data_ptr(), plen.data_ptr()))
    return score, cost, plen


def noalloc_status() -> int:
    """Device status of the fixed scratch after the last anomaly_score_noalloc
    on the current stream (0, WTS_EINVAL or WTS_ETIMEOUT; synchronises)."""
    s = ctypes.c_int32(0)
    check(_abi.load().wts_noalloc_read_status(_stream(), ctypes.byref(s)))
    return s.value


def dtw_align(B: torch.Tensor, batch: Batch, opts=None, ws: Workspace | None = None,
              jlo: torch.Tensor | None = None, jhi: torch.Tensor | None = None):
    """DTW and tie-rule path per cycle: (cost [T], plen [T], jlo [T, M], jhi [T, M]).
    jlo / jhi may be given (int32 [T, M], written in place); the ranges they
    hold on entry serve the walk as guesses (the previous call's paths)."""
    B = _check_B(B, batch.d)
    M = B.shape[0]
    lib = _abi.load()
    nb = workspace_size(_abi.OP_DTW_ALIGN, M, batch, opts)
    buf = _ws(ws, nb)
    dev = B.device
    cost = torch.empty(batch.T, dtype=torch.float32, device=dev)
    plen = torch.empty(batch.T, dtype=torch.int32, device=dev)
    for t in (jlo, jhi):
        if t is not None and not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()
                                  and tuple(t.shape) == (batch.T, M)):
            raise ValueError("jlo / jhi must be contiguous int32 CUDA tensors of shape [T, M]")
    jlo = torch.empty((batch.T, M), dtype=torch.int32, device=dev) if jlo is None else jlo
    jhi = torch.empty((batch.T, M), dtype=torch.int32, device=dev) if jhi is None else jhi
    check(lib.dtw_align(B.data_ptr(), M, ctypes.byref(batch.c()), _opt(opts), buf.data_ptr(), buf.numel(),
                        _stream(), cost.data_ptr(), plen.data_ptr(), jlo.data_ptr(), jhi.data_ptr()))
    return cost, plen, jlo, jhi


def subdtw_align(X: torch.Tensor, batch: Batch, opts=None, ws: Workspace | None = None):
    """Sub-DTW of X against every cycle (window) of the batch (Sec. 3.2):
    (cost [T], a_star [T], b_star [T], plen [T], jlo [T, M], jhi [T, M])."""
    X = _check_B(X, batch.d)
    M = X.shape[0]
    lib = _abi.load()
    nb = workspace_size(_abi.OP_SUBDTW, M, batch, opts)
    buf = _ws(ws, nb)
    dev = X.device
    cost = torch.empty(batch.T, dtype=torch.float32, device=dev)
    ab = torch.empty((3, batch.T), dtype=torch.int32, device=dev)
    jlo = torch.empty((batch.T, M), dtype=torch.int32, device=dev)
    jhi = torch.empty((batch.T, M), dtype=torch.int32, device=dev)
    check(lib.subdtw_align(X.data_ptr(), M, ctypes.byref(batch.c()), _opt(opts), buf.data_ptr(), buf.numel(),
                           _stream(), cost.data_ptr(), ab[0].data_ptr(), ab[1].data_ptr(), ab[2].data_ptr(),
                           jlo.data_ptr(), jhi.data_ptr()))
    return cost, ab[0], ab[1], ab[2], jlo, jhi


def segment(X: torch.Tensor, Y: torch.Tensor, alpha: int | None = None, opts=None, max_segments: int = 4096,
            ws: Workspace | None = None):
    """Cut the long series Y [N, d] (device) into cycles matching X [M, d]
    (Sec. 3.2; alpha None: the library's default 0.15 M).  Returns a list of
    (start, end, cost), inclusive bounds."""
    if Y.dim() == 1:
        Y = Y[:, None]
    if not (Y.is_cuda and Y.dtype == torch.float32 and Y.is_contiguous()):
        raise ValueError("Y must be a contiguous float32 CUDA tensor [N, d]")
    X = _check_B(X, Y.shape[1])
    M, d = X.shape
    N = Y.shape[0]
    if alpha is None:
        alpha = -1
    lib = _abi.load()
    nbytes = ctypes.c_size_t(0)
    check(lib.wts_segment_workspace_size(M, d, _opt(opts), ctypes.byref(nbytes)))
    buf = _ws(ws, nbytes.value)
    start = np.zeros(max_segments, dtype=np.int64)
    end = np.zeros(max_segments, dtype=np.int64)
    cost = np.zeros(max_segments, dtype=np.float32)
    n = ctypes.c_int32(0)
    check(lib.wts_segment(X.data_ptr(), M, Y.data_ptr(), N, d, alpha, _opt(opts), buf.data_ptr(), buf.numel(),
                          _stream(), max_segments, start.ctypes.data, end.ctypes.data, cost.ctypes.data,
                          ctypes.byref(n)))
    return [(int(start[k]), int(end[k]), float(cost[k])) for k in range(n.value)]


LBFGS_REASONS = {1: "gtol", 2: "ftol", 3: "max_iter", 4: "max_fun"}


def lbfgs_params(history=10, max_iter=40, max_fun=200, gtol=1e-8, ftol=1e-5, c1=1e-4):
    """L-BFGS settings; the defaults are Table I's (max iter 40, max fun 200,
    G tol 1e-8, tolerance 1e-5) with a history of 10 pairs."""
    p = _abi.wts_lbfgs_params()
    p.history, p.max_iter, p.max_fun = history, max_iter, max_fun
    p.gtol, p.ftol, p.c1 = gtol, ftol, c1
    return p


def lbfgs_minimize(fn, x0, params=None):
    """Minimise fn(x) -> (f, grad) from x0 with the library's L-BFGS (host).
    Returns (x, f, iterations, evaluations, reason)."""
    x = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).ravel().copy())
    n = x.size

    def cb(xp, fp, gp, ctx):
        xv = np.ctypeslib.as_array(xp, shape=(n,))
        f, g = fn(xv.copy())
        fp[0] = float(f)
        np.ctypeslib.as_array(gp, shape=(n,))[:] = np.asarray(g, dtype=np.float64).ravel()
        return 0

    cfn = _abi.OBJECTIVE_FN(cb)
    f = ctypes.c_double(0)
    it, ev, why = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    check(_abi.load().wts_lbfgs_minimize(n, x.ctypes.data, cfn, None, ctypes.byref(params or lbfgs_params()),
                                         ctypes.byref(f), ctypes.byref(it), ctypes.byref(ev), ctypes.byref(why)))
    return x.reshape(np.shape(x0)), f.value, it.value, ev.value, LBFGS_REASONS.get(why.value, why.value)


def softdtw_barycenter_lbfgs(batch: Batch, M: int, gamma: float, init: torch.Tensor | None = None,
                             weights: torch.Tensor | None = None, params=None, opts=None, ws: Workspace | None = None):
    """Soft-DTW barycenter (Eq. 7) by L-BFGS with Table I's settings: B
    minimises sum_k w_k Soft-DTW^gamma(B, Y_k), w_k = 1 / N_k unless given;
    starts from the Euclidean mean resampled to M unless ``init`` is given.
    Returns (B, objective, iterations, evaluations, stop reason)."""
    dev = batch.data.device
    B = euclid_mean(batch, M) if init is None else init.detach().clone().contiguous()
    lib = _abi.load()
    nb = workspace_size(_abi.OP_SOFTDTW_LBFGS, M, batch, opts)
    buf = _ws(ws, nb)
    f = ctypes.c_double(0)
    it, ev, why = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    check(lib.wts_softdtw_barycenter_lbfgs(B.data_ptr(), M, ctypes.byref(batch.c()), float(gamma),
                                           weights.data_ptr() if weights is not None else None,
                                           ctypes.byref(params or lbfgs_params()), _opt(opts), buf.data_ptr(),
                                           buf.numel(), _stream(), ctypes.byref(f), ctypes.byref(it),
                                           ctypes.byref(ev), ctypes.byref(why)))
    return B, f.value, it.value, ev.value, LBFGS_REASONS.get(why.value, why.value)


def thresholds(scores) -> tuple[float, float]:
    """The 2-sigma and boxplot detection thresholds of Sec. 5.3 on the scores
    (host computation in the library): (mean + 2 std, q3 + 1.5 |q3 - q1|)."""
    sc = np.ascontiguousarray(scores.detach().cpu().numpy() if isinstance(scores, torch.Tensor) else scores,
                              dtype=np.float32)
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    check(_abi.load().wts_thresholds(sc.ctypes.data, len(sc), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def f2_score(scores, labels, threshold: float) -> dict:
    """Confusion counts and F2 of "score > threshold" against labels (Sec. 5.3)."""
    sc = np.ascontiguousarray(scores.detach().cpu().numpy() if isinstance(scores, torch.Tensor) else scores,
                              dtype=np.float32)
    lb = np.ascontiguousarray((np.asarray(labels) != 0).astype(np.int8))
    tp, fp, fn = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    f2 = ctypes.c_double(0)
    check(_abi.load().wts_f2(sc.ctypes.data, lb.ctypes.data, len(sc), float(threshold), ctypes.byref(tp),
                             ctypes.byref(fp), ctypes.byref(fn), ctypes.byref(f2)))
    return {"tp": tp.value, "fp": fp.value, "fn": fn.value, "f2": f2.value}


def dba_iterate(B_in: torch.Tensor, batch: Batch, opts=None, ws: Workspace | None = None, B_out=None,
                counts=None, cost_before=None, cost=None):
    """One DBA iteration: (B_out [M, d], counts [M], cost_before (0-d float64), cost [T])."""
    B_in = _check_B(B_in, batch.d)
    M = B_in.shape[0]
    lib = _abi.load()
    nb = workspace_size(_abi.OP_DBA_ITERATE, M, batch, opts)
    buf = _ws(ws, nb)
    dev = B_in.device
    B_out = torch.empty_like(B_in) if B_out is None else B_out
    counts = torch.empty(M, dtype=torch.int32, device=dev) if counts is None else counts
    cost_before = torch.empty((), dtype=torch.float64, device=dev) if cost_before is None else cost_before
    cost = torch.empty(batch.T, dtype=torch.float32, device=dev) if cost is None else cost
    check(lib.dba_iterate(B_in.data_ptr(), B_out.data_ptr(), M, ctypes.byref(batch.c()), _opt(opts),
                          buf.data_ptr(), buf.numel(), _stream(), counts.data_ptr(), cost_before.data_ptr(),
                          cost.data_ptr()))
    return B_out, counts, cost_before, cost


def autotune(op: int, B: torch.Tensor, batch: Batch, ws: Workspace | None = None):
    """Time the candidate launch options of the wavefront for ``op`` on this
    batch and return (options, ms).  The workspace is sized for the largest
    candidate (for the score: also the form that walks stored codes)."""
    B = _check_B(B, batch.d)
    M = B.shape[0]
    forms = (0, 1) if op == _abi.OP_ANOMALY_SCORE else (0,)
    need = max(workspace_size(op, M, batch, options(rows_per_thread=r, score_via_codes=f))
               for r in ((8, 16, 32) if batch.d <= 3 else (8, 16)) for f in forms)
    buf = _ws(ws, need)
    best = wts_options()
    ms = ctypes.c_float(0)
    check(_abi.load().wts_autotune(op, B.data_ptr(), M, ctypes.byref(batch.c()), buf.data_ptr(), buf.numel(),
                                   _stream(), ctypes.byref(best), ctypes.byref(ms)))
    return best, ms.value


def capture(fn):
    """Capture fn() (library calls on the current stream) in a CUDA graph;
    returns (graph, fn's outputs).  Replaying the graph re-runs the calls on
    the same buffers."""
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn()                                # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        out = fn()
    return g, out


def compact_nan(batch: Batch, ws: Workspace | None = None) -> Batch:
    """Remove every time step with a NaN in any channel (Sec. 3.1) and re-pack:
    returns the compacted batch (its host offsets are read back, one sync)."""
    nb = workspace_size(_abi.OP_COMPACT_NAN, 0, batch)
    buf = _ws(ws, nb)
    out = torch.empty_like(batch.data)
    offs = torch.empty_like(batch.offsets)
    check(_abi.load().wts_compact_nan(ctypes.byref(batch.c()), buf.data_ptr(), buf.numel(), _stream(),
                                      out.data_ptr(), offs.data_ptr()))
    host = offs.cpu().numpy()
    return Batch(out[: int(host[-1])], offs, host)


def pad_last(batch: Batch, L: int = 0) -> Batch:
    """Sec. 4.1's equal-length form: every cycle extended with its last sample
    to length L (0: the longest cycle's); returns the padded batch of T cycles
    of length L."""
    Lh = int(batch.lengths.max()) if L == 0 else int(L)
    out = torch.empty((batch.T * Lh, batch.d), dtype=torch.float32, device=batch.data.device)
    check(_abi.load().wts_pad_last(ctypes.byref(batch.c()), int(L), _stream(), out.data_ptr()))
    offs_h = np.arange(batch.T + 1, dtype=np.int64) * Lh
    return Batch(out, torch.from_numpy(offs_h).to(batch.data.device), offs_h)


def select_channel(batch: Batch, c: int) -> Batch:
    """Channel c of every cycle as a d = 1 batch with the same offsets (the
    paper treats each joint on its own)."""
    out = torch.empty((batch.data.shape[0], 1), dtype=torch.float32, device=batch.data.device)
    check(_abi.load().wts_select_channel(ctypes.byref(batch.c()), int(c), _stream(), out.data_ptr()))
    return Batch(out, batch.offsets, batch.offsets_host)


def pairwise_dtw(batch: Batch, opts=None, ws: Workspace | None = None) -> torch.Tensor:
    """[T, T] symmetric matrix of DTW costs between cycles."""
    lib = _abi.load()
    nb = workspace_size(_abi.OP_PAIRWISE, 0, batch, opts)
    buf = _ws(ws, nb)
    C = torch.empty((batch.T, batch.T), dtype=torch.float32, device=batch.data.device)
    check(lib.wts_pairwise_dtw(ctypes.byref(batch.c()), _opt(opts), buf.data_ptr(), buf.numel(), _stream(),
                               C.data_ptr()))
    return C


def medoid(C: torch.Tensor):
    """(index (0-d int32 tensor), row sums [n] float64) of a pairwise cost matrix."""
    n = C.shape[0]
    sums = torch.empty(n, dtype=torch.float64, device=C.device)
    idx = torch.empty((), dtype=torch.int32, device=C.device)
    check(_abi.load().wts_medoid(C.contiguous().data_ptr(), n, _stream(), sums.data_ptr(), idx.data_ptr()))
    return idx, sums


def resample(x: torch.Tensor, M: int) -> torch.Tensor:
    if x.dim() == 1:
        x = x[:, None]
    x = x.contiguous()
    out = torch.empty((M, x.shape[1]), dtype=torch.float32, device=x.device)
    check(_abi.load().wts_resample(x.data_ptr(), x.shape[0], x.shape[1], out.data_ptr(), M, _stream()))
    return out


def euclid_mean(batch: Batch, M: int) -> torch.Tensor:
    out = torch.empty((M, batch.d), dtype=torch.float32, device=batch.data.device)
    check(_abi.load().wts_euclid_mean(ctypes.byref(batch.c()), M, out.data_ptr(), _stream()))
    return out


# --- Soft-DTW ------------------------------------------------------------------

def softdtw_forward(B: torch.Tensor, batch: Batch, gamma: float, opts=None, ws: Workspace | None = None):
    """Soft-DTW^gamma(B, Y_k) for every cycle (Eq. 4): values [T].  The
    workspace keeps R for softdtw_backward."""
    B = _check_B(B, batch.d)
    M = B.shape[0]
    nb = workspace_size(_abi.OP_SOFTDTW, M, batch, opts)
    buf = _ws(ws, nb)
    values = torch.empty(batch.T, dtype=torch.float32, device=B.device)
    check(_abi.load().softdtw_forward(B.data_ptr(), M, ctypes.byref(batch.c()), float(gamma), _opt(opts),
                                      buf.data_ptr(), buf.numel(), _stream(), values.data_ptr()))
    return values


def softdtw_backward(B: torch.Tensor, batch: Batch, gamma: float, grad_value: torch.Tensor | None = None,
                     opts=None, ws: Workspace | None = None, grad_B: torch.Tensor | None = None):
    """d/dB of sum_k grad_value[k] * Soft-DTW^gamma(B, Y_k) (Eq. 6): [M, d];
    grad_value None: the library's Eq. 7 weights 1 / N_k.  ``ws`` must be the
    workspace of the matching softdtw_forward."""
    B = _check_B(B, batch.d)
    M = B.shape[0]
    nb = workspace_size(_abi.OP_SOFTDTW, M, batch, opts)
    buf = _ws(ws, nb)
    gv = None
    if grad_value is not None:
        gv = grad_value.to(device=B.device, dtype=torch.float32).contiguous()
        if gv.numel() != batch.T:
            raise ValueError("grad_value must have T entries")
    grad_B = torch.empty_like(B) if grad_B is None else grad_B
    check(_abi.load().softdtw_backward(B.data_ptr(), M, ctypes.byref(batch.c()), float(gamma), _p(gv),
                                       _opt(opts), buf.data_ptr(), buf.numel(), _stream(), grad_B.data_ptr()))
    return grad_B


def adam_step(x: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, t: int,
              lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """In-place Adam update of x (library kernel)."""
    check(_abi.load().wts_adam_step(x.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), x.numel(),
                                    lr, beta1, beta2, eps, t, _stream()))


class SoftDTW(torch.autograd.Function):
    """values[k] = Soft-DTW^gamma(B, Y_k), differentiable in B through the
    hand-written backward kernel (each call owns its workspace, which holds R
    until backward)."""

    @staticmethod
    def forward(ctx, B, batch, gamma, opts=None):
        ws = Workspace(B.device)
        values = softdtw_forward(B.detach().contiguous(), batch, gamma, opts, ws)
        ctx.save_for_backward(B)
        ctx.batch, ctx.gamma, ctx.opts, ctx.ws = batch, gamma, opts, ws
        return values

    @staticmethod
    def backward(ctx, grad_values):
        (B,) = ctx.saved_tensors
        g = softdtw_backward(B.detach().contiguous(), ctx.batch, ctx.gamma, grad_values, ctx.opts, ctx.ws)
        return g, None, None, None


def softdtw(B: torch.Tensor, batch: Batch, gamma: float, opts=None) -> torch.Tensor:
    return SoftDTW.apply(B, batch, gamma, opts)


def softdtw_barycenter(batch: Batch, M: int, gamma: float, steps: int = 50, lr: float = 1e-2,
                       init: torch.Tensor | None = None, weights: torch.Tensor | None = None, opts=None,
                       beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, ws: Workspace | None = None):
    """Soft-DTW barycenter (Eq. 7) by Adam (the library's loop on the current
    stream): B minimises sum_k w_k Soft-DTW^gamma(B, Y_k), w_k = lambda_k / m_k
    (weights None: the library's 1 / N_k).  Starts from the Euclidean mean of
    the cycles resampled to M (Table I's default initialisation) unless
    ``init`` is given.  Returns (B, values per step [steps, T] on the device)."""
    dev = batch.data.device
    B = euclid_mean(batch, M) if init is None else init.detach().clone().contiguous()
    B = _check_B(B, batch.d)
    if weights is not None:
        weights = weights.to(device=dev, dtype=torch.float32).contiguous()
    nb = workspace_size(_abi.OP_SOFTDTW_ADAM, M, batch, opts)
    buf = _ws(ws if ws is not None else Workspace(dev), nb)
    hist = torch.empty((steps, batch.T), dtype=torch.float32, device=dev)
    check(_abi.load().wts_softdtw_barycenter_adam(B.data_ptr(), M, ctypes.byref(batch.c()), float(gamma), _p(weights),
                                                  int(steps), float(lr), float(beta1), float(beta2), float(eps),
                                                  _opt(opts), buf.data_ptr(), buf.numel(), _stream(),
                                                  hist.data_ptr() if steps > 0 else None))
    return B, hist

"""CPU oracle for the WETSAND alignment hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library (``paper_2404_12134_gb300``) and never imports
it; the only common module is the seeded input generator, which holds none of
the method's arithmetic.

What it computes (paper sections; the C body cites the equations):

* ``dtw``          - DTW cost, optimal path, per-row column ranges, |pi|
                     (Eq. 1, Eq. 5 at gamma = 0, Definitions "Alignment path"
                     and "Alignment matrix", Sec. 3.2);
* ``score``        - d_score = DTW / |pi| (Eq. 8, Sec. 3.4);
* ``dba_iterate``  - one DTW Barycenter Averaging step (cited in Sec. 2 and
                     used as a comparison in Table II; no formula printed);
* ``softdtw``      - Soft-DTW value, R, E and gradient (Eqs. 3-6);
* ``softdtw_batch``- barycenter objective Eq. 7 and its gradient;
* ``medoid``, ``resample``, ``euclid_mean`` - initial barycenters (Table I:
                     Euclidean-mean init; medoid for DBA);
* ``subdtw``, ``segment`` - Sub-DTW and the sliding-window segmentation into
                     cycles (Sec. 3.2);
* ``thresholds``, ``f2`` - the 2-sigma and boxplot detection thresholds and
                     the F2 score (Sec. 5.3).

``prec='f64'`` is the reference precision.  ``prec='f32'`` mirrors the CUDA
kernels' operation order in float so that the warping path, an integer
decision taken from float comparisons, is decided in the same precision on
both sides.

Parity status: every function is pinned by tests/test_oracle_pins.py against
brute-force enumeration, closed forms and invariants; the real-data
experiments of the paper (Tables II-VI) are not reproducible here (parity
unpinned for those, by absence of the data).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wetsand_oracle.c")
_HDR = os.path.join(_HERE, "oracle_body.h")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_libs: dict = {}

f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
VP = ctypes.c_void_p


def build(defines: tuple = (), force: bool = False) -> str:
    """Compile the oracle shared library (gcc, plain C, OpenMP across pairs)."""
    tag = "_".join(d.lower() for d in defines) or "plain"
    out = os.path.join(_BUILD, f"liboracle_{tag}.so")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"] + [f"-D{d}" for d in defines]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib(defines: tuple = ()):
    key = tuple(defines)
    with _lock:
        if key in _libs:
            return _libs[key]
        lib = ctypes.CDLL(build(key))
        for p, R, Rp in (("f64", ctypes.c_double, f64p), ("f32", ctypes.c_float, f32p)):
            fn = getattr(lib, f"orc_dtw_{p}")
            fn.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int,
                           VP, VP, VP, VP, VP, VP, ctypes.c_double, ctypes.c_int]
            fn.restype = ctypes.c_int
            fn = getattr(lib, f"orc_score_{p}")
            fn.argtypes = [f32p, ctypes.c_int64, f32p, i64p, ctypes.c_int, ctypes.c_int, VP, VP, VP, ctypes.c_double,
                           ctypes.c_int]
            fn.restype = ctypes.c_int
            fn = getattr(lib, f"orc_dba_{p}")
            fn.argtypes = [Rp, Rp, ctypes.c_int64, f32p, i64p, ctypes.c_int, ctypes.c_int, VP, VP, VP, ctypes.c_double,
                           ctypes.c_int]
            fn.restype = ctypes.c_int
            fn = getattr(lib, f"orc_softdtw_{p}")
            fn.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int, R, VP, VP, VP, VP, ctypes.c_double,
                           ctypes.c_int]
            fn.restype = ctypes.c_int
            fn = getattr(lib, f"orc_softdtw_batch_{p}")
            fn.argtypes = [f32p, ctypes.c_int64, f32p, i64p, ctypes.c_int, ctypes.c_int, R, VP, VP, VP, VP,
                           ctypes.c_double, ctypes.c_int]
            fn.restype = ctypes.c_int
            fn = getattr(lib, f"orc_subdtw_{p}")
            fn.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int64, ctypes.c_int, VP, VP, VP, VP, VP, VP, ctypes.c_int]
            fn.restype = ctypes.c_int
        _libs[key] = lib
        return lib


def _dt(prec: str):
    if prec not in ("f64", "f32"):
        raise ValueError(prec)
    return np.float64 if prec == "f64" else np.float32


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _as2d(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.float32)
    if x.ndim == 1:
        x = x[:, None]
    return np.ascontiguousarray(x)


def dtw(B, Y, prec: str = "f64", path: bool = True, band: float = 0.0, cost_kind: int = 0, _defines: tuple = ()):
    """DTW(B, Y) with its optimal path under the tie order diag > up > left.

    band > 0: Sakoe-Chiba band (Table I), cells with |i N - j M| > floor(band M N)
    excluded.  cost_kind 0: squared l2 local cost; 1: the l2 norm (Sec. 3.2).
    Returns dict(cost, plen, jlo, jhi, path_i, path_j); rows index B."""
    B = _as2d(B); Y = _as2d(Y)
    M, d = B.shape; N = Y.shape[0]
    assert Y.shape[1] == d and M >= 1 and N >= 1
    dt = _dt(prec)
    cost = np.zeros(1, dtype=dt)
    plen = np.zeros(1, dtype=np.int32)
    jlo = np.zeros(M, dtype=np.int32); jhi = np.zeros(M, dtype=np.int32)
    pi = np.zeros(M + N - 1, dtype=np.int32) if path else None
    pj = np.zeros(M + N - 1, dtype=np.int32) if path else None
    rc = getattr(_lib(_defines), f"orc_dtw_{prec}")(B, M, Y, N, d, _ptr(cost), _ptr(plen), _ptr(jlo), _ptr(jhi),
                                                  _ptr(pi), _ptr(pj), band, cost_kind)
    if rc:
        raise RuntimeError(f"oracle dtw failed (rc={rc}: -1 allocation, -2 invalid choice matrix, "
                           f"-3 band narrower than max(M, N))")
    L = int(plen[0])
    out = dict(cost=cost[0], plen=L, jlo=jlo, jhi=jhi)
    if path:
        out["path_i"] = pi[:L].copy(); out["path_j"] = pj[:L].copy()
    return out


def subdtw(X, Y, prec: str = "f64", cost_kind: int = 0, _defines: tuple = ()):
    """Sub-DTW(X, Y) (Sec. 3.2): min over a <= b of DTW(X, Y[a..b]).

    Returns dict(cost, a, b, plen, jlo, jhi): [a, b] is the matched piece of Y
    (0-based, inclusive; b the first end column of minimum cost), jlo/jhi the
    columns of each row of X on the path, plen = |pi|."""
    X = _as2d(X); Y = _as2d(Y)
    M, d = X.shape; N = Y.shape[0]
    assert Y.shape[1] == d and M >= 1 and N >= 1
    dt = _dt(prec)
    cost = np.zeros(1, dtype=dt)
    a = np.zeros(1, dtype=np.int32); b = np.zeros(1, dtype=np.int32); plen = np.zeros(1, dtype=np.int32)
    jlo = np.zeros(M, dtype=np.int32); jhi = np.zeros(M, dtype=np.int32)
    rc = getattr(_lib(_defines), f"orc_subdtw_{prec}")(X, M, Y, N, d, _ptr(cost), _ptr(a), _ptr(b), _ptr(plen),
                                                     _ptr(jlo), _ptr(jhi), cost_kind)
    if rc:
        raise RuntimeError(f"oracle subdtw failed (rc={rc})")
    return dict(cost=cost[0], a=int(a[0]), b=int(b[0]), plen=int(plen[0]), jlo=jlo, jhi=jhi)


def segment(X, Y, alpha: int, prec: str = "f32", cost_kind: int = 0):
    """Segmentation of a long series Y into cycles matching X (Sec. 3.2): the
    window [ws, ws + 2M) (cut at the end of Y) is aligned by Sub-DTW, the piece
    [ws + a*, ws + b*] is kept, and the next window starts at ws + b* - alpha,
    while ws < N.  Readings (the paper does not say): the window that reaches
    the end of Y is the last one (a later window would only cover its tail
    again), and when b* - alpha would not move the window forward the next one
    starts at ws + b* + 1.

    Returns a list of (start, end, cost) with inclusive 0-based bounds."""
    X = _as2d(X); Y = _as2d(Y)
    M = X.shape[0]; N = Y.shape[0]
    out = []
    ws = 0
    while ws < N:
        we = min(ws + 2 * M, N)
        r = subdtw(X, Y[ws:we], prec, cost_kind=cost_kind)
        a, b = ws + r["a"], ws + r["b"]
        out.append((a, b, r["cost"]))
        if we == N:
            break
        nxt = b - alpha
        ws = nxt if nxt > ws else b + 1
    return out


def score(B, data, offsets, prec: str = "f64", band: float = 0.0, cost_kind: int = 0, _defines: tuple = ()):
    """Similarity score Eq. 8 for each cycle of a packed batch: (score, cost, plen)."""
    B = _as2d(B); data = _as2d(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    T = offsets.shape[0] - 1
    dt = _dt(prec)
    s = np.zeros(T, dtype=dt); c = np.zeros(T, dtype=dt); L = np.zeros(T, dtype=np.int32)
    rc = getattr(_lib(_defines), f"orc_score_{prec}")(B, B.shape[0], data, offsets, T, B.shape[1],
                                                    _ptr(s), _ptr(c), _ptr(L), band, cost_kind)
    if rc:
        raise RuntimeError("oracle score failed (allocation, or a band narrower than max(M, N))")
    return s, c, L


def dba_iterate(B, data, offsets, prec: str = "f64", band: float = 0.0, cost_kind: int = 0, _defines: tuple = ()):
    """One DBA iteration: (B_new, counts, cost_before, per-cycle costs)."""
    dt = _dt(prec)
    B = np.ascontiguousarray(np.asarray(B, dtype=dt).reshape(len(B), -1))
    data = _as2d(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    T = offsets.shape[0] - 1
    M, d = B.shape
    Bo = np.zeros_like(B)
    cnt = np.zeros(M, dtype=np.int32)
    cb = np.zeros(1, dtype=np.float64)
    ck = np.zeros(T, dtype=dt)
    rc = getattr(_lib(_defines), f"orc_dba_{prec}")(B, Bo, M, data, offsets, T, d, _ptr(cnt), _ptr(cb), _ptr(ck),
                                                  band, cost_kind)
    if rc:
        raise RuntimeError("oracle dba failed (allocation, or a band narrower than max(M, N))")
    return Bo, cnt, float(cb[0]), ck


def softdtw(B, Y, gamma: float, prec: str = "f64", want_R=False, want_E=False, want_grad=True,
            band: float = 0.0, cost_kind: int = 0, _defines: tuple = ()):
    """Soft-DTW^gamma(B, Y), optionally R, E ((M+2) x (N+2), 1-based) and grad [M, d];
    band > 0: only the complete paths inside the Sakoe-Chiba band (as in ``dtw``);
    cost_kind as in ``dtw`` (1: the l2 norm, its gradient 0 where the norm is 0)."""
    B = _as2d(B); Y = _as2d(Y)
    M, d = B.shape; N = Y.shape[0]
    dt = _dt(prec)
    v = np.zeros(1, dtype=dt)
    R = np.zeros((M + 2, N + 2), dtype=dt) if want_R else None
    E = np.zeros((M + 2, N + 2), dtype=dt) if want_E else None
    g = np.zeros((M, d), dtype=dt) if want_grad else None
    rc = getattr(_lib(_defines), f"orc_softdtw_{prec}")(B, M, Y, N, d, gamma, _ptr(v), _ptr(R), _ptr(E), _ptr(g),
                                                      band, cost_kind)
    if rc:
        raise ValueError("oracle softdtw failed (allocation, gamma <= 0 with a gradient requested, "
                         "or a band narrower than max(M, N))")
    return dict(value=v[0], R=R, E=E, grad=g)


def softdtw_batch(B, data, offsets, gamma: float, weights=None, prec: str = "f64", want_grad=True,
                  band: float = 0.0, cost_kind: int = 0, _defines: tuple = ()):
    """Eq. 7 objective over a packed batch: (values[T], loss, grad[M, d] or None)."""
    B = _as2d(B); data = _as2d(data)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    T = offsets.shape[0] - 1
    M, d = B.shape
    dt = _dt(prec)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=dt)
    vals = np.zeros(T, dtype=dt)
    loss = np.zeros(1, dtype=dt)
    g = np.zeros((M, d), dtype=dt) if want_grad else None
    rc = getattr(_lib(_defines), f"orc_softdtw_batch_{prec}")(B, M, data, offsets, T, d, gamma, _ptr(w),
                                                            _ptr(vals), _ptr(loss), _ptr(g), band, cost_kind)
    if rc:
        raise ValueError("oracle softdtw_batch failed")
    return vals, loss[0], g


# --- initial barycenters (Table I: Euclidean-mean init; DBA: medoid) ---------

def medoid(data, offsets, subset=None, cost_kind: int = 0):
    """argmin_k sum_l DTW(Y_k, Y_l) over ``subset`` (default all); ties -> lowest k.

    Pairwise costs use the FP32 mirror (the same precision the GPU uses), the
    row sums are taken in double in ascending l.  Returns (index, cost matrix)."""
    data = _as2d(data)
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = np.arange(offsets.shape[0] - 1) if subset is None else np.asarray(subset)
    n = len(idx)
    C = np.zeros((n, n), dtype=np.float32)
    for a in range(n):
        for b in range(a + 1, n):
            ka, kb = int(idx[a]), int(idx[b])
            c = dtw(data[offsets[ka]:offsets[ka + 1]], data[offsets[kb]:offsets[kb + 1]], "f32", path=False,
                    cost_kind=cost_kind)["cost"]
            C[a, b] = C[b, a] = c
    sums = np.zeros(n, dtype=np.float64)
    for a in range(n):
        s = 0.0
        for b in range(n):
            s += float(C[a, b])
        sums[a] = s
    best = 0
    for a in range(1, n):
        if sums[a] < sums[best]:
            best = a
    return int(idx[best]), C


def resample(x, M: int) -> np.ndarray:
    """Linear resampling of a [N, d] series to M points spanning the same range.

    Position m maps to p = m (N - 1) / (M - 1) in double; the value is
    x[i] + (p - i)(x[i + 1] - x[i]) with i = floor(p), in double, rounded to float."""
    x = _as2d(x).astype(np.float64)
    N = x.shape[0]
    out = np.zeros((M, x.shape[1]), dtype=np.float64)
    for m in range(M):
        p = (m * (N - 1)) / (M - 1) if M > 1 else 0.0
        i = min(int(np.floor(p)), N - 1)
        f = p - i
        if i + 1 < N:
            out[m] = x[i] + f * (x[i + 1] - x[i])
        else:
            out[m] = x[i]
    return out.astype(np.float32)


def euclid_mean(data, offsets, M: int) -> np.ndarray:
    """Euclidean mean of the cycles, each resampled to M (Table I default init).
    Summed in double, k ascending, divided by T, rounded to float."""
    data = _as2d(data)
    offsets = np.asarray(offsets, dtype=np.int64)
    T = offsets.shape[0] - 1
    acc = np.zeros((M, data.shape[1]), dtype=np.float64)
    for k in range(T):
        acc += resample(data[offsets[k]:offsets[k + 1]], M).astype(np.float64)
    return (acc / T).astype(np.float32)


# --- the paper's own data forms ---------------------------------------------------

def pad_last(data, offsets, L: int = 0) -> np.ndarray:
    """Sec. 4.1: every cycle extended with its last sample to length L (0: the
    longest), as [T, L, d]."""
    data = _as2d(data)
    offsets = np.asarray(offsets, dtype=np.int64)
    T = offsets.shape[0] - 1
    n = np.diff(offsets)
    L = int(n.max()) if L == 0 else int(L)
    assert L >= n.max()
    out = np.zeros((T, L, data.shape[1]), dtype=np.float32)
    for k in range(T):
        for j in range(L):
            out[k, j] = data[offsets[k] + min(j, n[k] - 1)]
    return out


def select_channel(data, c: int) -> np.ndarray:
    """Channel c of every sample of a packed batch (each joint on its own, Sec. 5)."""
    return np.ascontiguousarray(_as2d(data)[:, c])


# --- detection thresholds (Sec. 5.3) ------------------------------------------

def thresholds(scores):
    """(2-sigma threshold, boxplot threshold) of Sec. 5.3: mean + 2 std (divisor
    T) and q3 + 1.5 |q3 - q1| with numpy's linear-interpolation quartiles."""
    x = np.asarray(scores, dtype=np.float64)
    q1, q3 = np.percentile(x, [25, 75])
    return float(x.mean() + 2.0 * x.std()), float(q3 + 1.5 * abs(q3 - q1))


def f2(scores, labels, threshold):
    """Confusion counts of score > threshold against labels and F2 = 5 TP / (5 TP + 4 FN + FP)."""
    flag = np.asarray(scores, dtype=np.float64) > threshold
    truth = np.asarray(labels) != 0
    tp = int((flag & truth).sum()); fp = int((flag & ~truth).sum()); fn = int((~flag & truth).sum())
    den = 5 * tp + 4 * fn + fp
    return {"tp": tp, "fp": fp, "fn": fn, "f2": 5 * tp / den if den else 0.0}


# --- L-BFGS (Table I's optimiser for the barycenter) ---------------------------

def lbfgs(fn, x0, history=10, max_iter=40, max_fun=200, gtol=1e-8, ftol=1e-5, c1=1e-4):
    """Limited-memory BFGS (two-loop recursion), restated from the standard
    method: d = -H g from the last ``history`` pairs with s.y > 0, scaled by
    (s.y)/(y.y) of the newest; no pair (or no descent): d = -g with a first
    step min(1, 1/||g||_2); backtracking from 1, halving until
    f(x + t d) <= f + c1 t g.d; stop at max|g| <= gtol ("gtol"), relative
    reduction <= ftol ("ftol"), max_iter, max_fun.
    Returns (x, f, iterations, evaluations, reason)."""
    x = np.asarray(x0, dtype=np.float64).ravel().copy()
    f, g = fn(x)
    g = np.asarray(g, dtype=np.float64).ravel()
    evals, it = 1, 0
    S, Y, rho = [], [], []
    while True:
        if np.max(np.abs(g)) <= gtol:
            why = "gtol"; break
        if it >= max_iter:
            why = "max_iter"; break
        q = g.copy()
        a = [0.0] * len(S)
        for k in range(len(S) - 1, -1, -1):
            a[k] = rho[k] * float(S[k] @ q)
            q -= a[k] * Y[k]
        if S:
            q *= float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
        for k in range(len(S)):
            bk = rho[k] * float(Y[k] @ q)
            q += S[k] * (a[k] - bk)
        d = -q
        gd = float(g @ d)
        t = 1.0
        if not S or not gd < 0:
            S, Y, rho = [], [], []
            d = -g
            gd = -float(g @ g)
            t = min(1.0, 1.0 / np.sqrt(-gd))
        accepted = False
        while evals < max_fun:
            xn = x + t * d
            fn_new, gn = fn(xn)
            gn = np.asarray(gn, dtype=np.float64).ravel()
            evals += 1
            if fn_new <= f + c1 * t * gd:
                accepted = True
                break
            t *= 0.5
        if not accepted:
            why = "max_fun"; break
        s, y = xn - x, gn - g
        sy = float(s @ y)
        if sy > 1e-10 * np.sqrt(float(s @ s) * float(y @ y)):
            if len(S) == history:
                S.pop(0); Y.pop(0); rho.pop(0)
            S.append(s); Y.append(y); rho.append(1.0 / sy)
        it += 1
        rel = (f - fn_new) / max(abs(f), abs(fn_new), 1.0)
        x, f, g = xn, fn_new, gn
        if rel <= ftol:
            why = "ftol"; break
    return x, f, it, evals, why


def softdtw_barycenter_lbfgs(data, offsets, B0, gamma: float, band: float = 0.0, cost_kind: int = 0, **params):
    """Eq. 7 barycenter by ``lbfgs``, the objective and gradient from
    ``softdtw_batch`` in FP64 at the float32 rounding of the iterate (the
    barycenter is a float32 array), weights 1 / N_k."""
    B0 = _as2d(B0)
    M, d = B0.shape
    lengths = np.diff(np.asarray(offsets, dtype=np.int64))
    w = (1.0 / lengths).astype(np.float32).astype(np.float64)

    def fn(x):
        Bf = x.reshape(M, d).astype(np.float32)
        vals, loss, g = softdtw_batch(Bf, data, offsets, gamma, weights=w, prec="f64", band=band,
                                      cost_kind=cost_kind)
        return float(loss), g.ravel()

    x, f, it, ev, why = lbfgs(fn, B0.astype(np.float64).ravel(), **params)
    return x.reshape(M, d).astype(np.float32), f, it, ev, why

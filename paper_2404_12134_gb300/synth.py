"""Seeded synthetic cycle generator.

The paper's workload is proprietary robot telemetry (quasi-periodic joint
signals with time warping and synchronous data gaps, Sec. 1.2 and Sec. 4.1);
it is not available, so every input here is synthetic and seeded.  This module
holds no step of the method's arithmetic (no cost, no recursion, no averaging):
it only draws signals.  Both the CUDA path and the CPU oracle are fed from it.

Recipe (the same text is kept in the design notes):

* base signal, single channel: 5 sinusoids (period = U(50, 400) samples of a
  1,100-sample reference cycle, amplitude U(0.2, 1), phase U(0, 2 pi)) plus 3
  ramps (height U(-1, 1), rising linearly over a random [t0, t1], held after),
  z-normalised on a 4,096-point grid;
* base signal, multichannel: per channel 8 Gaussian bumps (centre U(0, 1),
  width U(0.01, 0.08), amplitude N(0, 1)) plus 2 sinusoids (periods as above),
  z-normalised per channel;
* time warp: piecewise-linear monotone w: [0, 1] -> [0, 1] through 8 sorted
  U(0, 1) interior knots, segment slopes U(0.7, 1.4), renormalised to w(1) = 1;
  a cycle of pre-gap length L samples the base at w(n / L);
* noise N(0, 0.05^2) per sample and channel;
* gaps: 2 % of the samples removed as non-overlapping runs of U{5..20}
  samples, synchronous across channels (the NaN time steps that Sec. 3.1
  drops);
* anomalies: drift (a ramp 0 -> 0.5 std over a random 30 % window, held to the
  end), skipped segment (a random 5 % of base time is jumped over), slowdown
  (a random 10 % window of the warp runs 3x slower).

A batch is returned packed: ``data`` float32 [sum N_k, d] row-major,
``offsets`` int64 [T + 1], so cycle k is ``data[offsets[k]:offsets[k + 1]]``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 20240412
REF_CYCLE = 1100.0


@dataclasses.dataclass
class Batch:
    data: np.ndarray        # float32 [sum N_k, d]
    offsets: np.ndarray     # int64 [T + 1]
    labels: np.ndarray      # int8 [T]: 0 normal, 1 drift, 2 skip, 3 slowdown
    base: "BaseSignal"

    @property
    def T(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def d(self) -> int:
        return int(self.data.shape[1])

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def cycle(self, k: int) -> np.ndarray:
        return self.data[self.offsets[k]:self.offsets[k + 1]]

    def subset(self, idx) -> "Batch":
        cycles = [self.cycle(int(k)) for k in idx]
        return pack(cycles, self.labels[np.asarray(idx)], self.base)


class BaseSignal:
    """A smooth function of t in [0, 1) with d channels."""

    def __init__(self, rng: np.random.Generator, d: int, kind: str):
        self.d = d
        self.kind = kind
        if kind == "sines_ramps":
            assert d == 1
            self.per = rng.uniform(50, 400, size=(d, 5)) / REF_CYCLE
            self.amp = rng.uniform(0.2, 1.0, size=(d, 5))
            self.phase = rng.uniform(0, 2 * np.pi, size=(d, 5))
            t0 = rng.uniform(0, 1, size=(d, 3))
            t1 = rng.uniform(0, 1, size=(d, 3))
            self.r0 = np.minimum(t0, t1)
            self.r1 = np.maximum(t0, t1) + 1e-3
            self.rh = rng.uniform(-1, 1, size=(d, 3))
        elif kind == "bumps":
            self.centre = rng.uniform(0, 1, size=(d, 8))
            self.width = rng.uniform(0.01, 0.08, size=(d, 8))
            self.bamp = rng.normal(0, 1, size=(d, 8))
            self.per = rng.uniform(50, 400, size=(d, 2)) / REF_CYCLE
            self.amp = rng.uniform(0.2, 1.0, size=(d, 2))
            self.phase = rng.uniform(0, 2 * np.pi, size=(d, 2))
        else:
            raise ValueError(kind)
        grid = (np.arange(4096) + 0.5) / 4096
        raw = self._raw(grid)
        self.mu = raw.mean(axis=0)
        self.sd = raw.std(axis=0)

    def _raw(self, t: np.ndarray) -> np.ndarray:
        t = t[:, None, None]
        out = (self.amp * np.sin(2 * np.pi * t / self.per + self.phase)).sum(-1)
        if self.kind == "sines_ramps":
            frac = np.clip((t - self.r0) / (self.r1 - self.r0), 0.0, 1.0)
            out = out + (self.rh * frac).sum(-1)
        else:
            z = (t - self.centre) / self.width
            out = out + (self.bamp * np.exp(-0.5 * z * z)).sum(-1)
        return out

    def __call__(self, t: np.ndarray) -> np.ndarray:
        """[len(t), d] float64, z-normalised."""
        return (self._raw(np.asarray(t, dtype=np.float64)) - self.mu) / self.sd


def _warp(rng: np.random.Generator, slowdown: bool):
    """Knots (x, w(x)) of a monotone piecewise-linear warp with w(0)=0, w(1)=1."""
    xk = np.concatenate([[0.0], np.sort(rng.uniform(0, 1, 8)), [1.0]])
    slope = rng.uniform(0.7, 1.4, size=9)
    if slowdown:
        # a random 10 % window of cycle time runs 3x slower
        a = rng.uniform(0, 0.9)
        xs = np.unique(np.concatenate([xk, [a, a + 0.1]]))
        mid = 0.5 * (xs[:-1] + xs[1:])
        seg = np.clip(np.searchsorted(xk, mid, side="right") - 1, 0, 8)
        slope = np.where((mid > a) & (mid < a + 0.1), slope[seg] / 3.0, slope[seg])
        xk = xs
    wk = np.concatenate([[0.0], np.cumsum(slope * np.diff(xk))])
    wk = wk / wk[-1]
    return xk, wk


def _gaps(rng: np.random.Generator, L: int, frac: float = 0.02) -> np.ndarray:
    """Boolean keep-mask with about frac*L samples removed in runs of 5..20."""
    target = int(round(frac * L))
    runs = []
    tot = 0
    while tot < target:
        r = int(rng.integers(5, 21))
        runs.append(r)
        tot += r
    keep = np.ones(L, dtype=bool)
    if not runs or tot >= L:
        return keep
    pos = np.sort(rng.integers(0, L - tot + 1, size=len(runs)))
    shift = 0
    for p, r in zip(pos, runs):
        s = int(p) + shift
        keep[s:s + r] = False
        shift += r
    return keep


def make_cycle(rng: np.random.Generator, base: BaseSignal, L: int,
               anomaly: int = 0, noise: float = 0.05, gaps=True) -> np.ndarray:
    """One cycle of pre-gap length L: warp, optional anomaly, noise, gaps
    (gaps=True removes the missing steps, gaps="nan" keeps them as NaN rows, as
    a regularly sampled stream with missing values carries them)."""
    xk, wk = _warp(rng, slowdown=(anomaly == 3))
    x = np.arange(L) / L
    u = np.interp(x, xk, wk)
    if anomaly == 2:
        # skipped segment: 5 % of base time is jumped over
        a = rng.uniform(0, 0.95)
        u = u * 0.95
        u = np.where(u < a, u, u + 0.05)
    y = base(u)
    if anomaly == 1:
        a = rng.uniform(0, 0.7)
        ramp = np.clip((x - a) / 0.3, 0.0, 1.0) * 0.5
        y = y + ramp[:, None]
    y = y + rng.normal(0, noise, size=y.shape)
    if gaps == "nan":
        y = y.copy()
        y[~_gaps(rng, L)] = np.nan
    elif gaps:
        y = y[_gaps(rng, L)]
    return y.astype(np.float32)


def pack(cycles, labels=None, base=None) -> Batch:
    lengths = np.array([c.shape[0] for c in cycles], dtype=np.int64)
    offsets = np.zeros(len(cycles) + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    data = np.ascontiguousarray(np.concatenate(cycles, axis=0).astype(np.float32))
    if labels is None:
        labels = np.zeros(len(cycles), dtype=np.int8)
    return Batch(data=data, offsets=offsets, labels=np.asarray(labels, dtype=np.int8), base=base)


def make_batch(T: int, d: int, lengths, kind: str, seed: int,
               anomaly_frac: float = 0.0, anomaly_kinds=(1, 2),
               noise: float = 0.05, gaps: bool = True) -> Batch:
    """T cycles with pre-gap lengths ``lengths`` (array-like of T ints)."""
    rng = np.random.default_rng(seed)
    base = BaseSignal(rng, d, kind)
    lengths = np.asarray(lengths, dtype=np.int64)
    n_anom = int(round(anomaly_frac * T))
    labels = np.zeros(T, dtype=np.int8)
    if n_anom:
        idx = rng.choice(T, size=n_anom, replace=False)
        labels[idx] = rng.choice(np.asarray(anomaly_kinds), size=n_anom)
    cycles = [make_cycle(rng, base, int(lengths[k]), int(labels[k]), noise, gaps) for k in range(T)]
    return pack(cycles, labels, base)


# --- the five workload shapes -------------------------------------------------

def config_batch(cfg: int, scale: float = 1.0, T: int | None = None) -> Batch:
    """Synthetic batch shaped like workload ``cfg`` (0..4).

    ``scale`` shrinks every length (parity tests use small scales), ``T``
    overrides the cycle count.  Lengths are pre-gap.
    """
    rng = np.random.default_rng(SEED_BASE + 1000 + cfg)
    if cfg == 0:
        T = 16 if T is None else T
        lengths = rng.integers(1000, 1201, size=T)
        kind, d, af, ak = "sines_ramps", 1, 0.0, (1, 2)
    elif cfg == 1:
        T = 200 if T is None else T
        lengths = rng.integers(20000, 30001, size=T)
        kind, d, af, ak = "bumps", 6, 0.10, (1, 2)
    elif cfg == 2:
        T = 64 if T is None else T
        lengths = rng.integers(8000, 12001, size=T)
        kind, d, af, ak = "sines_ramps", 1, 0.0, (1, 2)
    elif cfg == 3:
        T = 1000 if T is None else T
        lengths = np.clip(np.exp(rng.normal(np.log(15000), 0.6, size=T)), 2000, 60000).astype(np.int64)
        kind, d, af, ak = "bumps", 3, 0.05, (1, 2, 3)
    elif cfg == 4:
        T = 32 if T is None else T
        lengths = rng.integers(100000, 120001, size=T)
        kind, d, af, ak = "bumps", 3, 0.0, (1, 2)
    else:
        raise ValueError(cfg)
    lengths = np.maximum(np.round(lengths * scale).astype(np.int64), 2)
    return make_batch(T, d, lengths, kind, SEED_BASE + cfg, af, ak)


PROTO_LEN = {0: None, 1: 25000, 2: 10000, 3: 20000, 4: 110000}


def segmentation_stream(K: int, lo: int, hi: int, d: int, ref_len: int, seed: int):
    """A long series of K back-to-back cycles (pre-gap lengths U{lo..hi}) of one
    multichannel base, each warped, noisy and with its own gaps removed, and a
    separately drawn reference cycle of pre-gap length ref_len (an operator's
    pick: warped, noisy, with gaps).  Returns (X [M, d], Y [N, d], bounds),
    bounds[k] = (first, last) sample of cycle k in Y (inclusive)."""
    rng = np.random.default_rng(seed)
    base = BaseSignal(rng, d, "bumps")
    X = make_cycle(rng, base, ref_len)
    cycles = [make_cycle(rng, base, int(rng.integers(lo, hi + 1))) for _ in range(K)]
    ends = np.cumsum([c.shape[0] for c in cycles])
    bounds = [(int(e - c.shape[0]), int(e - 1)) for e, c in zip(ends, cycles)]
    return X, np.ascontiguousarray(np.concatenate(cycles).astype(np.float32)), bounds


def clean_prototype(batch: Batch, M: int) -> np.ndarray:
    """The unwarped, noise-free base sampled at M points (fixed scoring prototype)."""
    return batch.base((np.arange(M) + 0.0) / M).astype(np.float32)


def integer_pair(rng: np.random.Generator, M: int, N: int, d: int, lo: int = -8, hi: int = 8):
    """Integer-valued samples: every cost is exact in FP32 and FP64, ties are common."""
    B = rng.integers(lo, hi + 1, size=(M, d)).astype(np.float32)
    Y = rng.integers(lo, hi + 1, size=(N, d)).astype(np.float32)
    return B, Y

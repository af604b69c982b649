"""Brute-force enumeration of complete alignment paths (tiny sizes only).

TEST INFRASTRUCTURE ONLY.  Independent of the oracle's recursion: it lists
every complete alignment path of Definition "Alignment path" (Sec. 3.2) and
evaluates Eq. 1 (min over paths of <A, Delta>) and Eq. 4 (soft-min over paths)
directly, plus the expected alignment matrix that the gradient Eq. 6 uses.
The number of paths is the Delannoy number D(M-1, N-1); keep M, N <= 6.
"""
from __future__ import annotations

import math

import numpy as np

# step codes of a path read backwards from (M-1, N-1): the ranking used by the
# tie rule (diag > up > left)
DIAG, UP, LEFT = 2, 1, 0


def delannoy(m: int, n: int) -> int:
    """D(m, n) = number of complete alignment paths of an (m+1) x (n+1) grid."""
    return sum(math.comb(m, k) * math.comb(n, k) * 2 ** k for k in range(min(m, n) + 1))


def paths(M: int, N: int):
    """All complete alignment paths from (0,0) to (M-1,N-1), as lists of cells."""
    out = []

    def rec(i, j, acc):
        if i == M - 1 and j == N - 1:
            out.append(list(acc))
            return
        for di, dj in ((0, 1), (1, 0), (1, 1)):
            a, b = i + di, j + dj
            if a < M and b < N:
                acc.append((a, b))
                rec(a, b, acc)
                acc.pop()

    rec(0, 0, [(0, 0)])
    return out


def cost_matrix(B, Y, cost_kind: int = 0) -> np.ndarray:
    """Delta[i, j] = sum_c (b_ic - y_jc)^2 in double (exact for small integers);
    cost_kind 1: the Euclidean norm, numpy's ``linalg.norm`` of b_i - y_j."""
    B = np.asarray(B, dtype=np.float64).reshape(len(B), -1)
    Y = np.asarray(Y, dtype=np.float64).reshape(len(Y), -1)
    if cost_kind:
        return np.linalg.norm(B[:, None, :] - Y[None, :, :], axis=-1)
    return ((B[:, None, :] - Y[None, :, :]) ** 2).sum(-1)


def reversed_steps(p):
    """Step codes of path p walked back from its end (for the tie rule)."""
    codes = []
    for k in range(len(p) - 1, 0, -1):
        (i1, j1), (i0, j0) = p[k], p[k - 1]
        di, dj = i1 - i0, j1 - j0
        codes.append(DIAG if (di, dj) == (1, 1) else UP if (di, dj) == (1, 0) else LEFT)
    return tuple(codes)


def dtw(B, Y, cost_kind: int = 0):
    """Eq. 1 by enumeration: (min cost, the tie-rule path, all optimal paths)."""
    D = cost_matrix(B, Y, cost_kind)
    M, N = D.shape
    ps = paths(M, N)
    costs = [sum(D[i, j] for i, j in p) for p in ps]
    best = min(costs)
    opt = [p for p, c in zip(ps, costs) if c == best]
    chosen = max(opt, key=reversed_steps)
    return best, chosen, opt


def softdtw(B, Y, gamma: float, cost_kind: int = 0):
    """Eq. 4 by enumeration: value -gamma log sum_A exp(-<A,Delta>/gamma) and the
    expected alignment matrix E = sum_A p(A) A, p(A) proportional to exp(-<A,Delta>/gamma)."""
    D = cost_matrix(B, Y, cost_kind)
    M, N = D.shape
    ps = paths(M, N)
    costs = np.array([sum(D[i, j] for i, j in p) for p in ps])
    m = costs.min()
    w = np.exp(-(costs - m) / gamma)
    Z = w.sum()
    value = m - gamma * math.log(Z)
    E = np.zeros((M, N))
    for p, wk in zip(ps, w):
        for i, j in p:
            E[i, j] += wk / Z
    return value, E


def subdtw(X, Y, cost_kind: int = 0):
    """Sub-DTW (Sec. 3.2) by enumeration over every piece Y[a..b] and every
    complete alignment path of X against it: (min cost, b*, the chosen path).

    b* is the smallest end column among the optimal pieces; the chosen path is,
    among the optimal paths ending at b*, the greatest under the tie order
    diag > up > left walked back from (M-1, b*), where leaving row 0 (the
    free start) counts as a diagonal step."""
    D = cost_matrix(X, Y, cost_kind)
    M, N = D.shape
    best = math.inf
    cands = []                      # (cost, b, path)
    for a in range(N):
        for b in range(a, N):
            for p in paths(M, b - a + 1):
                q = [(i, j + a) for i, j in p]
                c = sum(D[i, j] for i, j in q)
                cands.append((c, b, q))
                best = min(best, c)
    b_star = min(b for c, b, q in cands if c == best)
    opt = [q for c, b, q in cands if c == best and b == b_star]
    chosen = max(opt, key=lambda q: reversed_steps(q) + (DIAG,))
    return best, b_star, chosen


def in_band(i: int, j: int, M: int, N: int, band: float) -> bool:
    """Sakoe-Chiba band membership of 0-based cell (i, j): |i N - j M| <= floor(band M N)."""
    bound = math.floor(band * M * N)
    return abs(i * N - j * M) <= bound


def dtw_band(B, Y, band: float, cost_kind: int = 0):
    """Eq. 1 restricted to the complete paths that stay inside the band:
    (min cost, the tie-rule path)."""
    D = cost_matrix(B, Y, cost_kind)
    M, N = D.shape
    ps = [p for p in paths(M, N) if all(in_band(i, j, M, N, band) for i, j in p)]
    costs = [sum(D[i, j] for i, j in p) for p in ps]
    best = min(costs)
    chosen = max((p for p, c in zip(ps, costs) if c == best), key=reversed_steps)
    return best, chosen


def softdtw_band(B, Y, gamma: float, band: float, cost_kind: int = 0):
    """Eq. 4 over the complete paths inside the band: (value, E)."""
    D = cost_matrix(B, Y, cost_kind)
    M, N = D.shape
    ps = [p for p in paths(M, N) if all(in_band(i, j, M, N, band) for i, j in p)]
    costs = np.array([sum(D[i, j] for i, j in p) for p in ps])
    m = costs.min()
    w = np.exp(-(costs - m) / gamma)
    Z = w.sum()
    E = np.zeros((M, N))
    for p, wk in zip(ps, w):
        for i, j in p:
            E[i, j] += wk / Z
    return m - gamma * math.log(Z), E

"""A model, in plain Python, of the segmented backtrack's rounds (the order of
the rounds, the guessed starts, the stop where a re-walk enters its previous
walk, the final check that the segments join up), run against the one-walk
backtrack on random code matrices.  Within a round the segments are taken
in a random order, as the warps of one launch may be.  No GPU."""
import random

import numpy as np

DIAG, UP, LEFT = 0, 1, 2


def _move(code, i, j):
    """(di, dj) of the stored code of cell (i, j): diag, up or left."""
    c = code[i][j]
    return (1, 1) if c == DIAG else ((1, 0) if c == UP else (0, 1))


def one_walk(code, M, N):
    """The plain walk from (M-1, N-1): (|pi| or -1, jlo, jhi)."""
    i, j, ln = M - 1, N - 1, 0
    jlo, jhi = {}, {M - 1: j}
    while True:
        ln += 1
        if i == 0 and j == 0:
            break
        di, dj = _move(code, i, j)
        if (i == 0 and di) or (j == 0 and dj):
            return -1, jlo, jhi
        if di:
            jlo[i] = j
            jhi[i - 1] = j - dj
        i -= di
        j -= dj
    jlo[0] = 0
    return ln, jlo, jhi


def segmented_walk(code, M, N, S, arrays_jhi, rng):
    """The rounds of the segmented walk over segments of S rows."""
    nseg = (M + S - 1) // S
    jlo, jhi = {}, dict(arrays_jhi)          # the range arrays hold old contents
    start = [None] * nseg
    exit_ = [[None, None] for _ in range(nseg)]
    status = [0] * nseg
    for rnd in range(nseg):
        cur = rnd & 1
        last_exit = [e[1 - cur] for e in exit_]
        order = list(range(nseg))
        rng.shuffle(order)
        for k in order:
            top, lo = min(M, (k + 1) * S) - 1, k * S
            if top == M - 1:
                if rnd > 0:
                    exit_[k][cur] = exit_[k][1 - cur]
                    continue
                s = N - 1
            elif rnd == 0:
                s = jhi.get(top, -1)
                if not 0 <= s < N:
                    s = top * (N - 1) // max(M - 1, 1)
            else:
                s = last_exit[k + 1]
                if s == start[k]:
                    exit_[k][cur] = exit_[k][1 - cur]
                    continue
            if s is None or not 0 <= s < N:
                start[k], exit_[k][cur], status[k] = s, -1, 1
                continue
            mergeable = rnd > 0 and status[k] == 0
            prev_exit = exit_[k][1 - cur]
            if mergeable and jlo[top] <= s <= start[k]:
                jhi[top], start[k], exit_[k][cur] = s, s, prev_exit
                continue
            i, j, ln = top, s, 0
            jhi[i], start[k] = j, s
            left = merged = False
            while True:
                ln += 1
                if i == 0 and j == 0:
                    break
                di, dj = _move(code, i, j)
                if (i == 0 and di) or (j == 0 and dj):
                    ln = -1
                    break
                if di and mergeable and i - 1 >= lo and jlo[i - 1] <= j - dj <= jhi[i - 1]:
                    jlo[i], jhi[i - 1] = j, j - dj
                    merged = True
                    break
                if di:
                    jlo[i], jhi[i - 1] = j, j - dj
                i -= di
                j -= dj
                if i < lo:
                    left = True
                    break
            if merged:
                exit_[k][cur] = prev_exit
                continue
            exit_[k][cur] = j if left else -1
            status[k] = 1 if ln < 0 else 0
            if not left and i == 0 and j == 0 and ln > 0:
                jlo[0] = 0
    fin = (nseg - 1) & 1
    bad = any(status) or any(start[k] != exit_[k + 1][fin] for k in range(nseg - 1))
    plen = -1 if bad else sum(jhi[i] - jlo[i] + 1 for i in range(M))
    return plen, jlo, jhi


def test_segmented_rounds_reproduce_the_walk():
    rng = np.random.default_rng(7)
    order_rng = random.Random(11)
    for trial in range(600):
        M, N = int(rng.integers(1, 70)), int(rng.integers(1, 70))
        p = rng.dirichlet([1, 1, 1]) if trial % 2 else [0.8, 0.1, 0.1]
        code = rng.choice(3, size=(M, N), p=p).tolist()
        if trial % 13:
            # a complete DP's codes: only up on column 0, only left on row 0
            for i in range(1, M):
                code[i][0] = UP
            for j in range(1, N):
                code[0][j] = LEFT
        S = int(rng.integers(1, 20))
        hint = {i: int(rng.integers(-3, N + 3)) for i in range(M)} if trial % 3 else {}
        want = one_walk(code, M, N)
        got = segmented_walk(code, M, N, S, hint, order_rng)
        if want[0] < 0:
            assert got[0] == -1, trial
            continue
        assert got[0] == want[0], trial
        assert all(got[1][i] == want[1][i] for i in range(M)), trial
        assert all(got[2][i] == want[2][i] for i in range(M)), trial

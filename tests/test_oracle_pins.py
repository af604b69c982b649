"""Pins of the CPU oracle against things other than itself.

Each check ties the oracle to brute-force enumeration over all alignment paths
(Definition "Alignment path", Eq. 1, Eq. 4), to a closed form, or to an
invariant of the mathematics; none re-derives the oracle's recursion.  The
last test plants plausible mistakes in the oracle (compile-time mutation
hooks) and checks that each one trips at least one pin.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_2404_12134_gb300 import synth


def _real_pair(rng, M, N, d):
    return (rng.normal(size=(M, d)).astype(np.float32), rng.normal(size=(N, d)).astype(np.float32))


# --- DTW: brute force -------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dtw_matches_brute_force_integer_ties(prec):
    """Integer samples in {-3..3}: every cost exact, ties frequent.  Cost equal,
    and the path equal to the lexicographically greatest optimal path under
    the tie order diag > up > left."""
    rng = np.random.default_rng(11)
    for M in range(1, 7):
        for N in range(1, 7):
            for d in (1, 2, 3):
                B, Y = synth.integer_pair(rng, M, N, d, -3, 3)
                best, chosen, opt = brute.dtw(B, Y)
                r = oracle.dtw(B, Y, prec)
                assert float(r["cost"]) == best, (M, N, d)
                assert list(zip(r["path_i"].tolist(), r["path_j"].tolist())) == chosen, (M, N, d)
                assert r["plen"] == len(chosen)


def test_dtw_matches_brute_force_real():
    rng = np.random.default_rng(12)
    for M in range(1, 7):
        for N in range(1, 7):
            B, Y = _real_pair(rng, M, N, 2)
            best, chosen, opt = brute.dtw(B, Y)
            r = oracle.dtw(B, Y, "f64")
            assert abs(r["cost"] - best) <= 1e-12 * max(1.0, best)
            assert list(zip(r["path_i"].tolist(), r["path_j"].tolist())) == chosen


def test_path_counts_are_delannoy():
    # the enumerator itself: number of complete paths = Delannoy D(M-1, N-1)
    for M in range(1, 7):
        for N in range(1, 7):
            assert len(brute.paths(M, N)) == brute.delannoy(M - 1, N - 1)
    assert brute.delannoy(5, 5) == 1683


# --- DTW: closed forms and invariants ----------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_dtw_self_is_zero_on_diagonal(prec):
    rng = np.random.default_rng(13)
    x = rng.normal(size=(257, 3)).astype(np.float32)
    r = oracle.dtw(x, x, prec)
    assert r["cost"] == 0
    assert r["plen"] == 257
    assert (r["path_i"] == np.arange(257)).all() and (r["path_j"] == np.arange(257)).all()
    assert (r["jlo"] == np.arange(257)).all() and (r["jhi"] == np.arange(257)).all()


def test_dtw_symmetric_cost():
    rng = np.random.default_rng(14)
    for M, N in ((40, 55), (1, 9), (9, 1), (63, 64)):
        B, Y = _real_pair(rng, M, N, 3)
        a = oracle.dtw(B, Y, "f64")["cost"]
        b = oracle.dtw(Y, B, "f64")["cost"]
        assert abs(a - b) <= 1e-12 * max(1.0, abs(a))
        Bi, Yi = synth.integer_pair(rng, M, N, 2)
        assert oracle.dtw(Bi, Yi, "f32")["cost"] == oracle.dtw(Yi, Bi, "f32")["cost"]


def test_dtw_bounded_by_euclidean_for_equal_lengths():
    rng = np.random.default_rng(15)
    for M in (1, 5, 100):
        B, Y = _real_pair(rng, M, M, 2)
        euc = float(((B.astype(np.float64) - Y) ** 2).sum())
        assert oracle.dtw(B, Y, "f64")["cost"] <= euc * (1 + 1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_single_row_and_single_column_closed_form(prec):
    rng = np.random.default_rng(16)
    x = rng.integers(-5, 6, size=(1, 2)).astype(np.float32)
    Y = rng.integers(-5, 6, size=(37, 2)).astype(np.float32)
    exact = float(((Y.astype(np.float64) - x) ** 2).sum())
    r = oracle.dtw(x, Y, prec)
    assert float(r["cost"]) == exact and r["plen"] == 37
    assert r["jlo"][0] == 0 and r["jhi"][0] == 36
    r = oracle.dtw(Y, x, prec)
    assert float(r["cost"]) == exact and r["plen"] == 37
    assert (r["jlo"] == 0).all() and (r["jhi"] == 0).all()


def test_integer_inputs_f32_equals_f64():
    """Integer samples keep every partial sum exact in float and double, so the
    two precisions must agree bit for bit, ties included."""
    rng = np.random.default_rng(17)
    for M, N, d in ((200, 180, 3), (64, 300, 1), (129, 130, 6)):
        B, Y = synth.integer_pair(rng, M, N, d)
        a = oracle.dtw(B, Y, "f64"); b = oracle.dtw(B, Y, "f32")
        assert float(a["cost"]) == float(b["cost"])
        assert (a["path_i"] == b["path_i"]).all() and (a["path_j"] == b["path_j"]).all()


def test_ranges_describe_the_path():
    rng = np.random.default_rng(18)
    B, Y = _real_pair(rng, 90, 140, 2)
    r = oracle.dtw(B, Y, "f64")
    jlo, jhi = r["jlo"], r["jhi"]
    assert jlo[0] == 0 and jhi[-1] == 139
    assert (jlo <= jhi).all()
    assert ((jlo[1:] == jhi[:-1]) | (jlo[1:] == jhi[:-1] + 1)).all()
    assert int((jhi - jlo + 1).sum()) == r["plen"]
    # |pi| = M + N - 1 - number of diagonal steps
    di = np.diff(r["path_i"]); dj = np.diff(r["path_j"])
    assert r["plen"] == 90 + 140 - 1 - int(((di == 1) & (dj == 1)).sum())


# --- score (Eq. 8) ------------------------------------------------------------

def test_score_closed_forms():
    rng = np.random.default_rng(19)
    x = rng.normal(size=(50, 2)).astype(np.float32)
    Y = rng.normal(size=(70, 2)).astype(np.float32)
    data = np.concatenate([x, Y]); offs = np.array([0, 50, 120])
    s, c, L = oracle.score(x, data, offs, "f64")
    assert s[0] == 0 and L[0] == 50
    # single-sample prototype: score = mean local cost
    s, c, L = oracle.score(x[:1], data, offs, "f64")
    mean = ((Y.astype(np.float64) - x[0]) ** 2).sum(-1).mean()
    assert abs(s[1] - mean) <= 1e-12 * mean and L[1] == 70


# --- DBA ----------------------------------------------------------------------

def test_dba_cost_non_increasing():
    b = synth.config_batch(0, scale=0.08)
    k0, _ = oracle.medoid(b.data, b.offsets)
    B = b.cycle(k0).astype(np.float64)
    prev = math.inf
    for _ in range(8):
        B, cnt, cost, _ = oracle.dba_iterate(B, b.data, b.offsets, "f64")
        assert cost <= prev * (1 + 1e-12)
        prev = cost


def test_dba_counts_and_average_against_brute_force_paths():
    rng = np.random.default_rng(20)
    T, M, d = 3, 5, 2
    B = rng.normal(size=(M, d)).astype(np.float32)
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in (4, 6, 5)]
    data = np.concatenate(cyc); offs = np.array([0, 4, 10, 15])
    Bn, cnt, cost, ck = oracle.dba_iterate(B, data, offs, "f64")
    sums = np.zeros((M, d)); n = np.zeros(M)
    tot = 0.0
    for y in cyc:
        best, path, _ = brute.dtw(B, y)
        tot += best
        for i, j in path:
            sums[i] += y[j]; n[i] += 1
    assert (cnt == n).all() and (cnt >= T).all()
    assert np.allclose(Bn, sums / n[:, None], rtol=0, atol=1e-12)
    assert abs(cost - tot) <= 1e-12 * tot


def test_dba_fixed_points():
    rng = np.random.default_rng(21)
    x = rng.normal(size=(40, 3)).astype(np.float32)
    data = np.concatenate([x, x, x]); offs = np.array([0, 40, 80, 120])
    Bn, cnt, cost, _ = oracle.dba_iterate(x, data, offs, "f32")
    assert (Bn == x).all() and cost == 0 and (cnt == 3).all()
    const = np.full((33, 3), 0.375, dtype=np.float32)
    data = np.concatenate([const, const[:20], const[:27]]); offs = np.array([0, 33, 53, 80])
    Bn, cnt, cost, _ = oracle.dba_iterate(rng.normal(size=(25, 3)), data, offs, "f64")
    assert (Bn == 0.375).all()


# --- Soft-DTW ------------------------------------------------------------------

def test_softdtw_matches_brute_force():
    rng = np.random.default_rng(22)
    for M in range(1, 6):
        for N in range(1, 6):
            B, Y = _real_pair(rng, M, N, 2)
            for g in (0.1, 1.0, 10.0):
                v, E = brute.softdtw(B, Y, g)
                r = oracle.softdtw(B, Y, g, "f64", want_E=True)
                assert abs(r["value"] - v) <= 1e-10 * max(1.0, abs(v)), (M, N, g)
                assert np.allclose(r["E"][1:M + 1, 1:N + 1], E, rtol=1e-9, atol=1e-12), (M, N, g)


def test_softdtw_sandwich_and_limit():
    """DTW - gamma ln D(M-1,N-1) <= Soft-DTW <= DTW, so Soft-DTW -> DTW as gamma -> 0."""
    rng = np.random.default_rng(23)
    B, Y = _real_pair(rng, 6, 6, 1)
    dtw = oracle.dtw(B, Y, "f64")["cost"]
    nA = brute.delannoy(5, 5)
    for g in (1.0, 0.1, 0.01, 0.001):
        v = oracle.softdtw(B, Y, g, "f64", want_grad=False)["value"]
        assert dtw - g * math.log(nA) - 1e-12 <= v <= dtw + 1e-12
    B, Y = _real_pair(rng, 60, 70, 2)
    dtw = oracle.dtw(B, Y, "f64")["cost"]
    assert oracle.softdtw(B, Y, 0.0, "f64", want_grad=False)["value"] == dtw


def test_softdtw_E_properties():
    rng = np.random.default_rng(24)
    B, Y = _real_pair(rng, 30, 41, 2)
    E = oracle.softdtw(B, Y, 0.5, "f64", want_E=True)["E"][1:31, 1:42]
    assert (E >= 0).all() and (E <= 1 + 1e-12).all()
    assert abs(E[0, 0] - 1) < 1e-12 and abs(E[-1, -1] - 1) < 1e-12
    assert (E.sum(1) >= 1 - 1e-9).all() and (E.sum(0) >= 1 - 1e-9).all()


@pytest.mark.parametrize("gamma", [0.1, 1.0])
def test_softdtw_gradient_finite_differences(gamma):
    """Central differences, h = 1e-3, lengths <= 64, in double."""
    rng = np.random.default_rng(25)
    B, Y = _real_pair(rng, 24, 64, 2)
    g = oracle.softdtw(B, Y, gamma, "f64")["grad"]
    h = 1e-3
    for (i, c) in ((0, 0), (5, 1), (23, 0), (12, 1)):
        Bp = B.astype(np.float64).copy(); Bm = Bp.copy()
        # the oracle takes float32 samples: perturb by a float-representable step
        Bp[i, c] += h; Bm[i, c] -= h
        vp = oracle.softdtw(Bp.astype(np.float32), Y, gamma, "f64", want_grad=False)["value"]
        vm = oracle.softdtw(Bm.astype(np.float32), Y, gamma, "f64", want_grad=False)["value"]
        hp = float(np.float32(Bp[i, c])) - float(np.float32(Bm[i, c]))
        fd = (vp - vm) / hp
        assert abs(fd - g[i, c]) <= 1e-4 * max(1.0, abs(g[i, c])), (i, c, fd, g[i, c])


def test_softdtw_batch_objective():
    rng = np.random.default_rng(26)
    B = rng.normal(size=(12, 1)).astype(np.float32)
    cyc = [rng.normal(size=(n, 1)).astype(np.float32) for n in (10, 14, 9)]
    data = np.concatenate(cyc); offs = np.array([0, 10, 24, 33])
    vals, loss, grad = oracle.softdtw_batch(B, data, offs, 0.3)
    exp_loss = 0.0; exp_grad = np.zeros_like(grad)
    for y in cyc:
        r = oracle.softdtw(B, y, 0.3)
        exp_loss += r["value"] / len(y); exp_grad += r["grad"] / len(y)
    assert abs(loss - exp_loss) < 1e-12 and np.allclose(grad, exp_grad, atol=1e-12)
    # gradient of the objective by central differences
    h = 1e-3
    Bp = B.copy(); Bp[4, 0] += np.float32(h)
    Bm = B.copy(); Bm[4, 0] -= np.float32(h)
    fd = (oracle.softdtw_batch(Bp, data, offs, 0.3, want_grad=False)[1]
          - oracle.softdtw_batch(Bm, data, offs, 0.3, want_grad=False)[1]) / (float(Bp[4, 0]) - float(Bm[4, 0]))
    assert abs(fd - grad[4, 0]) < 1e-4 * max(1, abs(grad[4, 0]))


# --- init helpers ---------------------------------------------------------------

def test_resample_and_mean():
    x = np.arange(10, dtype=np.float32)[:, None] * 2 + 1
    assert (oracle.resample(x, 10) == x).all()
    y = oracle.resample(x, 19)           # a line stays a line, endpoints kept
    assert y[0, 0] == 1 and y[-1, 0] == 19 and np.allclose(np.diff(y[:, 0]), 1.0)
    data = np.concatenate([x, x + 2]); offs = np.array([0, 10, 20])
    assert np.allclose(oracle.euclid_mean(data, offs, 10), x + 1)


def test_medoid_brute_force():
    rng = np.random.default_rng(27)
    cyc = [rng.normal(size=(n, 1)).astype(np.float32) for n in (5, 4, 6, 5)]
    cyc.append(cyc[0] * 0 + cyc[3].mean())     # a flat cycle
    data = np.concatenate(cyc); offs = np.concatenate([[0], np.cumsum([len(c) for c in cyc])])
    k, C = oracle.medoid(data, offs)
    S = [sum(brute.dtw(a, b)[0] for b in cyc) for a in cyc]
    assert k == int(np.argmin(S))


def test_generator_is_seeded():
    a = synth.config_batch(1, scale=0.01); b = synth.config_batch(1, scale=0.01)
    assert (a.data == b.data).all() and (a.offsets == b.offsets).all()
    assert a.d == 6 and a.T == 200 and int(a.labels.astype(bool).sum()) == 20


# --- Sakoe-Chiba band (Table I) ----------------------------------------------------

def _bands(M, N):
    """Band widths from the narrowest accepted (floor(w M N) = max(M, N)) up to no restriction."""
    lo = max(M, N) / (M * N)
    return [lo * f for f in (1.0, 1.3, 2.0)] + [0.6, 1.0]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_banded_dtw_matches_brute_force(prec):
    """Integer samples; every band from the narrowest accepted one up: the cost
    and the tie-rule path over the complete paths that stay in the band."""
    rng = np.random.default_rng(50)
    for M in range(1, 7):
        for N in range(1, 7):
            B, Y = synth.integer_pair(rng, M, N, 2, -3, 3)
            for w in _bands(M, N):
                if math.floor(w * M * N) < max(M, N):
                    continue
                best, chosen = brute.dtw_band(B, Y, w)
                r = oracle.dtw(B, Y, prec, band=w)
                assert float(r["cost"]) == best, (M, N, w)
                assert list(zip(r["path_i"].tolist(), r["path_j"].tolist())) == chosen, (M, N, w)


def test_banded_softdtw_matches_brute_force():
    """Soft-DTW restricted to the in-band paths: value and E against
    enumeration, for the narrowest accepted band and a wider one; E is zero
    outside the band."""
    rng = np.random.default_rng(53)
    for M, N in ((4, 6), (6, 3), (5, 5), (3, 3)):
        B, Y = _real_pair(rng, M, N, 2)
        for w in (max(M, N) / (M * N), 0.45):
            if math.floor(w * M * N) < max(M, N):
                continue
            for gamma in (1.0, 0.3):
                v, E = brute.softdtw_band(B, Y, gamma, w)
                r = oracle.softdtw(B, Y, gamma, "f64", want_E=True, band=w)
                assert abs(r["value"] - v) <= 1e-10 * max(1.0, abs(v)), (M, N, w, gamma)
                assert np.allclose(r["E"][1:M + 1, 1:N + 1], E, atol=1e-10), (M, N, w, gamma)
    # w >= 1 is no band
    B, Y = _real_pair(rng, 30, 41, 1)
    a = oracle.softdtw(B, Y, 0.5, "f64")
    b = oracle.softdtw(B, Y, 0.5, "f64", band=1.0)
    assert a["value"] == b["value"] and np.array_equal(a["grad"], b["grad"])


def test_band_limits_and_refusal():
    """w >= 1 changes nothing; the cost never decreases as the band narrows;
    M = N with floor(w N^2) = N is the band |i - j| <= 1; a band narrower than
    max(M, N) is refused."""
    rng = np.random.default_rng(51)
    for M, N in ((40, 40), (37, 61), (70, 23)):
        B, Y = _real_pair(rng, M, N, 2)
        full = oracle.dtw(B, Y, "f64")
        assert oracle.dtw(B, Y, "f64", band=1.0)["cost"] == full["cost"]
        prev = full["cost"]
        for w in (0.6, 0.3, 0.1, max(M, N) / (M * N)):
            c = oracle.dtw(B, Y, "f64", band=w)["cost"]
            assert c >= prev
            prev = c
    B, Y = _real_pair(rng, 30, 30, 1)
    r = oracle.dtw(B, Y, "f64", band=30 / 900)
    assert all(abs(i - j) <= 1 for i, j in zip(r["path_i"], r["path_j"]))
    with pytest.raises(RuntimeError):
        oracle.dtw(B, Y, "f64", band=29 / 900)


def test_planted_band_mistake_is_caught():
    """The band written with the lengths swapped (|i M - j N|) trips the
    brute-force pin (it differs only when M != N)."""
    def fails(defines):
        rng = np.random.default_rng(52)
        for M, N in ((3, 5), (5, 2), (4, 6)):
            B, Y = synth.integer_pair(rng, M, N, 1, -3, 3)
            w = 1.3 * max(M, N) / (M * N)
            best, chosen = brute.dtw_band(B, Y, w)
            try:
                r = oracle.dtw(B, Y, "f64", band=w, _defines=defines)
            except RuntimeError:
                return True
            if float(r["cost"]) != best or list(zip(r["path_i"].tolist(), r["path_j"].tolist())) != chosen:
                return True
        return False
    assert not fails(())
    assert fails(("ORACLE_PLANT_BAND_SWAP",))


# --- Sub-DTW and segmentation (Sec. 3.2) ---------------------------------------

def _path_of(r):
    """Cells of the oracle's Sub-DTW path from its per-row column ranges."""
    cells = []
    for i in range(len(r["jlo"])):
        cells += [(i, j) for j in range(int(r["jlo"][i]), int(r["jhi"][i]) + 1)]
    return cells


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_subdtw_matches_brute_force(prec):
    """Integer samples (exact costs, frequent ties): the minimum over every
    piece Y[a..b] and every path, the first optimal end column, and the path
    chosen by the tie order."""
    rng = np.random.default_rng(40)
    for M in range(1, 5):
        for N in range(1, 7):
            for d in (1, 2):
                X, Y = synth.integer_pair(rng, M, N, d, -2, 2)
                best, b_star, chosen = brute.subdtw(X, Y)
                r = oracle.subdtw(X, Y, prec)
                assert float(r["cost"]) == best, (M, N, d)
                assert r["b"] == b_star and r["a"] == chosen[0][1], (M, N, d)
                assert _path_of(r) == chosen and r["plen"] == len(chosen), (M, N, d)


def test_subdtw_real_values_brute_force():
    rng = np.random.default_rng(41)
    for M, N in ((3, 6), (4, 5), (2, 6)):
        X, Y = _real_pair(rng, M, N, 2)
        best, b_star, chosen = brute.subdtw(X, Y)
        r = oracle.subdtw(X, Y, "f64")
        assert abs(r["cost"] - best) <= 1e-12 * max(1.0, best)
        assert r["b"] == b_star and _path_of(r) == chosen


def test_subdtw_embedded_copy_and_bounds():
    """X copied exactly into Y between samples far from it: cost 0 on the
    copy, one cell per row.  In general Sub-DTW <= DTW(X, Y), and with one
    column the cost is sum_i delta(i, 0)."""
    rng = np.random.default_rng(42)
    X = rng.normal(size=(37, 3)).astype(np.float32)
    pre = (rng.normal(size=(23, 3)) + 20).astype(np.float32)
    post = (rng.normal(size=(41, 3)) - 20).astype(np.float32)
    Y = np.concatenate([pre, X, post])
    for prec in ("f64", "f32"):
        r = oracle.subdtw(X, Y, prec)
        assert float(r["cost"]) == 0.0 and (r["a"], r["b"]) == (23, 23 + 36) and r["plen"] == 37
        assert (r["jlo"] == np.arange(23, 60)).all() and (r["jhi"] == r["jlo"]).all()
    for _ in range(5):
        X, Y = _real_pair(rng, 17, 29, 2)
        assert oracle.subdtw(X, Y)["cost"] <= oracle.dtw(X, Y, path=False)["cost"] + 1e-12
        y = Y[5:6]
        r = oracle.subdtw(X, y)
        assert abs(r["cost"] - brute.cost_matrix(X, y)[:, 0].sum()) <= 1e-12 * r["cost"]
        assert (r["a"], r["b"], r["plen"]) == (0, 0, 17)


def test_segmentation_of_repeated_copies():
    """A series of K exact copies of X: every window holds one whole copy at
    zero cost, so the first K pieces are the copies themselves; the loop ends
    once the window start passes the end of the series."""
    rng = np.random.default_rng(43)
    M, K = 29, 6
    X = rng.normal(size=(M, 2)).astype(np.float32)
    Y = np.concatenate([X] * K)
    segs = oracle.segment(X, Y, alpha=int(0.15 * M))
    assert [(a, b) for a, b, c in segs[:K]] == [(k * M, k * M + M - 1) for k in range(K)]
    assert all(float(c) == 0.0 for a, b, c in segs[:K])
    assert all(b < len(Y) for a, b, c in segs)


def pieces_match_cycles(segs, bounds, min_found):
    """Each piece lies (>= 95 % of its samples) inside one generated cycle and
    covers >= 90 % of it; pieces come in order, one per cycle; at least
    min_found cycles are found.  (A cycle may be skipped: the window can hold
    two cycles and Sub-DTW keeps the cheaper one, leaving the fragment before
    a* unassigned, as Sec. 3.2 notes.)"""
    hit = []
    for a, b, c in segs:
        best = max(range(len(bounds)), key=lambda k: min(b, bounds[k][1]) - max(a, bounds[k][0]))
        s0, s1 = bounds[best]
        ov = min(b, s1) - max(a, s0) + 1
        assert ov >= 0.95 * (b - a + 1) and ov >= 0.90 * (s1 - s0 + 1), ((a, b), (s0, s1))
        hit.append(best)
    assert hit == sorted(set(hit)) and len(hit) >= min_found, hit


def test_segmentation_recovers_generated_cycles():
    """A stream of K warped, noisy, gapped cycles of one base, segmented with a
    separately drawn reference cycle; the generator's bounds are the ground
    truth, independent of the oracle."""
    for d, seed in ((3, 7), (9, 8), (1, 9)):
        X, Y, bounds = synth.segmentation_stream(6, 550, 650, d, 600, seed)
        segs = oracle.segment(X, Y, int(0.15 * len(X)), "f32")
        pieces_match_cycles(segs, bounds, len(bounds) - 1)


def _sub_pins_fail(defines) -> bool:
    rng = np.random.default_rng(44)
    try:
        for M in range(1, 4):
            for N in range(2, 6):
                X, Y = synth.integer_pair(rng, M, N, 1, -2, 2)
                best, b_star, chosen = brute.subdtw(X, Y)
                r = oracle.subdtw(X, Y, "f64", _defines=defines)
                if float(r["cost"]) != best or r["b"] != b_star or _path_of(r) != chosen:
                    return True
    except Exception:
        return True
    return False


@pytest.mark.parametrize("plant", ["ORACLE_PLANT_SUB_FIXED_START", "ORACLE_PLANT_SUB_LAST_END"])
def test_planted_subdtw_mistakes_are_caught(plant):
    assert not _sub_pins_fail(())
    assert _sub_pins_fail((plant,))


# --- mutation check: each planted mistake trips a pin ----------------------------

def _pins_fail(defines) -> bool:
    rng = np.random.default_rng(28)
    try:
        for M in range(2, 7):
            for N in range(2, 7):
                for d in (1, 3):
                    B, Y = synth.integer_pair(rng, M, N, d, -2, 2)
                    best, chosen, _ = brute.dtw(B, Y)
                    r = oracle.dtw(B, Y, "f64", _defines=defines)
                    if float(r["cost"]) != best or list(zip(r["path_i"].tolist(), r["path_j"].tolist())) != chosen:
                        return True
        for M, N in ((4, 5), (6, 3), (5, 5)):
            B, Y = _real_pair(rng, M, N, 2)
            v, E = brute.softdtw(B, Y, 0.5)
            s = oracle.softdtw(B, Y, 0.5, "f64", want_E=True, _defines=defines)
            if abs(s["value"] - v) > 1e-9 * max(1, abs(v)) or not np.allclose(s["E"][1:M + 1, 1:N + 1], E, atol=1e-9):
                return True
    except Exception:
        return True
    return False


@pytest.mark.parametrize("plant", ["ORACLE_PLANT_DROP_CHANNEL", "ORACLE_PLANT_DIAG_INDEX",
                                   "ORACLE_PLANT_TIE_ORDER", "ORACLE_PLANT_SOFTMIN_SIGN",
                                   "ORACLE_PLANT_E_TRANSPOSE"])
def test_planted_mistakes_are_caught(plant):
    assert not _pins_fail(())
    assert _pins_fail((plant,))


# --- the l2-norm local cost (cost_kind 1, Sec. 3.2's "Euclidean distance") -----

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_l2_dtw_matches_brute_force_integer_ties(prec):
    """d = 1 integer samples: the l2 norm is |b - y|, an exact integer, so every
    path cost is exact and ties are frequent; cost and tie-rule path equal to
    the enumeration's (numpy's norm)."""
    rng = np.random.default_rng(61)
    for M in range(1, 7):
        for N in range(1, 7):
            B, Y = synth.integer_pair(rng, M, N, 1, -3, 3)
            best, chosen, _ = brute.dtw(B, Y, cost_kind=1)
            r = oracle.dtw(B, Y, prec, cost_kind=1)
            assert float(r["cost"]) == best, (M, N)
            assert list(zip(r["path_i"].tolist(), r["path_j"].tolist())) == chosen, (M, N)
            assert r["plen"] == len(chosen)


def test_l2_dtw_matches_brute_force_real():
    """d = 2, 3 real samples: cost within rounding; the path equal wherever the
    optimum is unique by a margin."""
    rng = np.random.default_rng(62)
    for M in range(1, 7):
        for N in range(1, 7):
            for d in (2, 3):
                B, Y = _real_pair(rng, M, N, d)
                best, chosen, _ = brute.dtw(B, Y, cost_kind=1)
                r = oracle.dtw(B, Y, "f64", cost_kind=1)
                assert abs(r["cost"] - best) <= 1e-12 * max(1.0, best), (M, N, d)
                D = brute.cost_matrix(B, Y, 1)
                costs = sorted(sum(D[i, j] for i, j in p) for p in brute.paths(M, N))
                if len(costs) == 1 or costs[1] - costs[0] > 1e-9:
                    assert list(zip(r["path_i"].tolist(), r["path_j"].tolist())) == chosen, (M, N, d)


def test_l2_closed_forms():
    """One row: DTW = sum_j ||b - y_j||.  DTW(x, x) = 0.  Equal lengths: DTW <=
    sum_i ||x_i - y_i|| (the diagonal path).  Samples in {0, 1} with d = 1:
    |b - y| = (b - y)^2, so both costs agree, paths included."""
    rng = np.random.default_rng(63)
    b = rng.normal(size=(1, 3)).astype(np.float32)
    Y = rng.normal(size=(17, 3)).astype(np.float32)
    want = float(np.linalg.norm(b.astype(np.float64) - Y.astype(np.float64), axis=1).sum())
    assert abs(oracle.dtw(b, Y, "f64", cost_kind=1)["cost"] - want) <= 1e-12 * want
    X = rng.normal(size=(40, 2)).astype(np.float32)
    assert oracle.dtw(X, X, "f64", cost_kind=1)["cost"] == 0.0
    Z = rng.normal(size=(40, 2)).astype(np.float32)
    diag = float(np.linalg.norm(X.astype(np.float64) - Z.astype(np.float64), axis=1).sum())
    assert oracle.dtw(X, Z, "f64", cost_kind=1)["cost"] <= diag + 1e-12
    for _ in range(10):
        B = rng.integers(0, 2, size=(9, 1)).astype(np.float32)
        Y = rng.integers(0, 2, size=(12, 1)).astype(np.float32)
        a, s = oracle.dtw(B, Y, "f32", cost_kind=1), oracle.dtw(B, Y, "f32")
        assert a["cost"] == s["cost"] and (a["jlo"] == s["jlo"]).all() and (a["jhi"] == s["jhi"]).all()


def test_l2_subdtw_matches_brute_force():
    rng = np.random.default_rng(64)
    for M in range(1, 4):
        for N in range(1, 6):
            X, Y = synth.integer_pair(rng, M, N, 1, -3, 3)
            best, b_star, chosen = brute.subdtw(X, Y, cost_kind=1)
            r = oracle.subdtw(X, Y, "f32", cost_kind=1)
            assert float(r["cost"]) == best and r["b"] == b_star and _path_of(r) == chosen, (M, N)


def test_l2_dba_against_brute_force_paths():
    """The DBA update under the l2 alignment: each row's mean of the samples
    that the brute-force tie-rule paths associate with it."""
    rng = np.random.default_rng(65)
    B = rng.integers(-3, 4, size=(5, 1)).astype(np.float32)
    cyc = [rng.integers(-3, 4, size=(n, 1)).astype(np.float32) for n in (6, 4, 5)]
    data = np.concatenate(cyc); offs = np.array([0, 6, 10, 15])
    sums = np.zeros((5, 1)); cnt = np.zeros(5, dtype=np.int64); total = 0.0
    for y in cyc:
        best, chosen, _ = brute.dtw(B, y, cost_kind=1)
        total += best
        for i, j in chosen:
            sums[i] += y[j]; cnt[i] += 1
    Bo, counts, cb, _ = oracle.dba_iterate(B, data, offs, "f64", cost_kind=1)
    assert (counts == cnt).all() and cb == total
    assert np.allclose(Bo, sums / cnt[:, None], rtol=0, atol=1e-15)


def test_l2_softdtw_matches_brute_force():
    rng = np.random.default_rng(66)
    for M in range(1, 6):
        for N in range(1, 6):
            B, Y = _real_pair(rng, M, N, 2)
            for g in (0.1, 1.0):
                v, E = brute.softdtw(B, Y, g, cost_kind=1)
                r = oracle.softdtw(B, Y, g, "f64", want_E=True, cost_kind=1)
                assert abs(r["value"] - v) <= 1e-10 * max(1.0, abs(v)), (M, N, g)
                assert np.allclose(r["E"][1:M + 1, 1:N + 1], E, rtol=1e-9, atol=1e-12), (M, N, g)


@pytest.mark.parametrize("gamma", [0.1, 1.0])
def test_l2_softdtw_gradient_finite_differences(gamma):
    """Central differences of the l2 objective (every distance > 0 for normal
    samples): d ||b - y|| / d b = (b - y) / ||b - y||, no factor 2."""
    rng = np.random.default_rng(67)
    B, Y = _real_pair(rng, 20, 48, 3)
    g = oracle.softdtw(B, Y, gamma, "f64", cost_kind=1)["grad"]
    h = 1e-3
    for (i, c) in ((0, 0), (7, 2), (19, 1), (11, 0)):
        Bp = B.astype(np.float64).copy(); Bm = Bp.copy()
        Bp[i, c] += h; Bm[i, c] -= h
        vp = oracle.softdtw(Bp.astype(np.float32), Y, gamma, "f64", want_grad=False, cost_kind=1)["value"]
        vm = oracle.softdtw(Bm.astype(np.float32), Y, gamma, "f64", want_grad=False, cost_kind=1)["value"]
        hp = float(np.float32(Bp[i, c])) - float(np.float32(Bm[i, c]))
        fd = (vp - vm) / hp
        assert abs(fd - g[i, c]) <= 1e-4 * max(1.0, abs(g[i, c])), (i, c, fd, g[i, c])
    # B = Y: every diagonal distance is 0, where the norm has no derivative;
    # the gradient takes 0 there and stays finite
    X = rng.normal(size=(10, 2)).astype(np.float32)
    assert np.isfinite(oracle.softdtw(X, X, gamma, "f64", cost_kind=1)["grad"]).all()


def _l2_pins_fail(defines) -> bool:
    rng = np.random.default_rng(68)
    try:
        for M in range(2, 6):
            for N in range(2, 6):
                B, Y = synth.integer_pair(rng, M, N, 1, -3, 3)
                best, chosen, _ = brute.dtw(B, Y, cost_kind=1)
                r = oracle.dtw(B, Y, "f64", cost_kind=1, _defines=defines)
                if float(r["cost"]) != best:
                    return True
        B, Y = _real_pair(rng, 12, 20, 2)
        g = oracle.softdtw(B, Y, 0.5, "f64", cost_kind=1, _defines=defines)["grad"]
        h = 1e-3
        Bp = B.astype(np.float64).copy(); Bm = Bp.copy()
        Bp[3, 1] += h; Bm[3, 1] -= h
        vp = oracle.softdtw(Bp.astype(np.float32), Y, 0.5, "f64", want_grad=False, cost_kind=1,
                            _defines=defines)["value"]
        vm = oracle.softdtw(Bm.astype(np.float32), Y, 0.5, "f64", want_grad=False, cost_kind=1,
                            _defines=defines)["value"]
        fd = (vp - vm) / (float(np.float32(Bp[3, 1])) - float(np.float32(Bm[3, 1])))
        if abs(fd - g[3, 1]) > 1e-4 * max(1.0, abs(g[3, 1])):
            return True
    except Exception:
        return True
    return False


@pytest.mark.parametrize("plant", ["ORACLE_PLANT_L2_NO_SQRT", "ORACLE_PLANT_L2_GRAD_TWO"])
def test_planted_l2_mistakes_are_caught(plant):
    assert not _l2_pins_fail(())
    assert _l2_pins_fail((plant,))


# --- the paper's data forms: last-value padding (Sec. 4.1), one joint (Sec. 5) --

def test_pad_last_and_select_channel():
    """Padding: the first N_k rows are the cycle, the rest repeat its last
    sample; an equal-length batch is unchanged; DTW against a prototype whose
    last sample equals the cycle's is unchanged by the padding (the extra
    columns align to the last row at cost 0, and folding them back onto column
    N gives a path of the unpadded pair that costs no more).  Channel
    selection: the channels stacked back give the batch."""
    rng = np.random.default_rng(71)
    cyc = [rng.normal(size=(n, 3)).astype(np.float32) for n in (5, 9, 1, 7)]
    data = np.concatenate(cyc); offs = np.array([0, 5, 14, 15, 22])
    P = oracle.pad_last(data, offs)
    assert P.shape == (4, 9, 3)
    for k, y in enumerate(cyc):
        assert (P[k, :len(y)] == y).all() and (P[k, len(y):] == y[-1]).all()
    P12 = oracle.pad_last(data, offs, 12)
    assert P12.shape == (4, 12, 3) and (P12[:, :9] == P).all()
    eq = np.concatenate([rng.normal(size=(6, 2)).astype(np.float32) for _ in range(3)])
    assert (oracle.pad_last(eq, np.array([0, 6, 12, 18])).reshape(-1, 2) == eq).all()
    assert (np.stack([oracle.select_channel(data, c) for c in range(3)], 1) == data).all()
    # DTW is unchanged by last-value padding when the prototype ends at the
    # cycle's last value (the extra columns align to the last row at cost 0)
    B = np.concatenate([rng.normal(size=(6, 3)).astype(np.float32), cyc[1][-1:]])
    assert oracle.dtw(B, P[1][:9], "f64")["cost"] == oracle.dtw(B, cyc[1], "f64")["cost"]
    assert oracle.dtw(B, P12[1], "f64")["cost"] == oracle.dtw(B, cyc[1], "f64")["cost"]


def test_l2_with_band_matches_brute_force():
    """Both options at once: the l2-norm cost inside the Sakoe-Chiba band,
    DTW (d = 1 integers, exact) and Soft-DTW (value and E) against the
    enumeration of the in-band paths."""
    rng = np.random.default_rng(69)
    for M in range(2, 6):
        for N in range(2, 6):
            for w in _bands(M, N)[:3]:
                B, Y = synth.integer_pair(rng, M, N, 1, -3, 3)
                best, chosen = brute.dtw_band(B, Y, w, cost_kind=1)
                r = oracle.dtw(B, Y, "f64", band=w, cost_kind=1)
                assert float(r["cost"]) == best, (M, N, w)
                assert list(zip(r["path_i"].tolist(), r["path_j"].tolist())) == chosen, (M, N, w)
                Br, Yr = _real_pair(rng, M, N, 2)
                v, E = brute.softdtw_band(Br, Yr, 0.5, w, cost_kind=1)
                s = oracle.softdtw(Br, Yr, 0.5, "f64", want_E=True, band=w, cost_kind=1)
                assert abs(s["value"] - v) <= 1e-10 * max(1.0, abs(v)), (M, N, w)
                assert np.allclose(s["E"][1:M + 1, 1:N + 1], E, rtol=1e-9, atol=1e-12), (M, N, w)

"""GPU parity of Soft-DTW forward / backward (Eqs. 3-7) against the oracle,
through the C ABI, plus the autograd wrapper and the Adam barycenter.

Tolerances, derived from the arithmetic:
* values: within 1e-5 of the FP64 oracle, relative to max(|value|, 1)
  (the 1e-5 relative bar of the target; the floor 1 keeps the bar
  meaningful for values near 0, which are differences of path sums; the
  measured error is below 1.1e-6);
* gradients: the exponent of every weight exp(((r(s) - r) - delta(s))/gamma)
  carries the FP32 rounding of r, of order ulp(r)/gamma, so no fixed relative
  bound holds at small gamma or large r.  The bar is that the kernel adds
  nothing beyond that: its error against the FP64 oracle (infinity norm,
  relative) is at most twice that of the same recursion evaluated in plain
  FP32 by the oracle's FP32 mode, plus 1e-5.
"""
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


VALUE_TOL = 1e-5


def _grad_bar(B, b, gamma, weights, go):
    """Twice the relative error of a plain FP32 evaluation, plus 1e-5."""
    g32 = oracle.softdtw_batch(B, b.data, b.offsets, gamma, weights=weights.astype(np.float32), prec="f32")[2]
    return 2.0 * np.abs(g32.astype(np.float64) - go).max() / np.abs(go).max() + 1e-5


def _case(seed, M, lens, d):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(M, d)).astype(np.float32)
    cyc = [rng.normal(size=(n, d)).astype(np.float32) for n in lens]
    return B, synth.pack(cyc)


CASES = [
    (1, 5, [1, 2, 7], 1),
    (2, 64, [64, 40, 100], 1),
    (3, 300, [1, 31, 33, 257, 700], 1),
    (4, 513, [400, 600], 3),
    (5, 260, [650, 80], 6),
    (6, 520, [300, 777], 2),
]


@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
@pytest.mark.parametrize("case", CASES, ids=[f"M{c[1]}-d{c[3]}" for c in CASES])
def test_softdtw_value_and_gradient(wts, case, gamma):
    seed, M, lens, d = case
    B, b = _case(seed, M, lens, d)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    v = wts.softdtw_forward(Bt, gb, gamma, ws=ws)
    w = torch.from_numpy((1.0 / np.asarray(lens)).astype(np.float32)).cuda()
    g = wts.softdtw_backward(Bt, gb, gamma, w, ws=ws)
    assert wts.read_status(ws.buf) == 0
    vo, lo, go = oracle.softdtw_batch(B, b.data, b.offsets, gamma, weights=1.0 / np.asarray(lens, dtype=np.float64))
    vg = v.cpu().numpy().astype(np.float64)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(vg - vo) <= VALUE_TOL * np.maximum(np.abs(vo), 1.0)), np.abs(vg - vo).max()
    err = np.abs(gg - go).max() / np.abs(go).max()
    assert err <= _grad_bar(B, b, gamma, 1.0 / np.asarray(lens, dtype=np.float64), go), err


def test_gradient_against_finite_differences(wts):
    """Central differences (h = 1e-3) of the FP64 oracle's Eq. 7 objective, lengths <= 64."""
    B, b = _case(7, 48, [64, 50, 33], 1)
    gamma = 0.1
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    wts.softdtw_forward(Bt, gb, gamma, ws=ws)
    w = torch.from_numpy((1.0 / b.lengths).astype(np.float32)).cuda()
    g = wts.softdtw_backward(Bt, gb, gamma, w, ws=ws).cpu().numpy()
    for i in (0, 11, 30, 47):
        Bp = B.copy(); Bp[i, 0] += np.float32(1e-3)
        Bm = B.copy(); Bm[i, 0] -= np.float32(1e-3)
        fp = oracle.softdtw_batch(Bp, b.data, b.offsets, gamma, want_grad=False)[1]
        fm = oracle.softdtw_batch(Bm, b.data, b.offsets, gamma, want_grad=False)[1]
        fd = (fp - fm) / (float(Bp[i, 0]) - float(Bm[i, 0]))
        assert abs(fd - g[i, 0]) <= 2e-3 * max(1.0, abs(fd)), (i, fd, g[i, 0])


def test_autograd_function(wts):
    B, b = _case(8, 100, [90, 120], 2)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    vals = wts.softdtw(Bt, gb, 0.5)
    w = torch.tensor([0.3, -1.7], device="cuda")
    (vals * w).sum().backward()
    vo, lo, go = oracle.softdtw_batch(B, b.data, b.offsets, 0.5, weights=np.array([0.3, -1.7]))
    err = np.abs(Bt.grad.cpu().numpy() - go).max() / np.abs(go).max()
    assert err <= _grad_bar(B, b, 0.5, np.array([0.3, -1.7]), go)


def test_soft_barycenter_decreases_objective(wts):
    """Eq. 7 by Adam from the Euclidean-mean init: the objective, evaluated by
    the FP64 oracle, drops."""
    b = synth.config_batch(2, scale=0.02, T=8)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M = 200
    B0 = wts.euclid_mean(gb, M)
    B, hist = wts.softdtw_barycenter(gb, M, gamma=0.1, steps=30, lr=2e-2, init=B0)
    f0 = oracle.softdtw_batch(B0.cpu().numpy(), b.data, b.offsets, 0.1, want_grad=False)[1]
    f1 = oracle.softdtw_batch(B.cpu().numpy(), b.data, b.offsets, 0.1, want_grad=False)[1]
    assert f1 < f0
    w = (1.0 / b.lengths).astype(np.float32)
    h = (hist.cpu().numpy().astype(np.float64) * w).sum(1)
    assert h[-1] < h[0]


@pytest.mark.parametrize("explicit_weights", [False, True])
def test_adam_barycenter_call_equals_primitive_loop(wts, explicit_weights):
    """wts_softdtw_barycenter_adam (the library's own loop) equals, bit for
    bit, the same steps driven one C-ABI call at a time: softdtw_forward,
    softdtw_backward with the weights (NULL: the library's 1 / N_k), and
    wts_adam_step.  Also: NULL weights give exactly the FP32 1 / N_k."""
    b = synth.config_batch(2, scale=0.03, T=6)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M, gamma, steps, lr = 300, 0.1, 7, 3e-2
    B0 = wts.euclid_mean(gb, M)
    w = torch.from_numpy((1.0 / b.lengths).astype(np.float32)).cuda()
    B, hist = wts.softdtw_barycenter(gb, M, gamma, steps=steps, lr=lr, init=B0,
                                     weights=w if explicit_weights else None)
    Bp = B0.clone()
    m = torch.zeros_like(Bp)
    v = torch.zeros_like(Bp)
    ws = wts.Workspace()
    grad = torch.empty_like(Bp)
    hp = []
    for t in range(1, steps + 1):
        hp.append(wts.softdtw_forward(Bp, gb, gamma, ws=ws))
        wts.softdtw_backward(Bp, gb, gamma, w, ws=ws, grad_B=grad)
        g_null = wts.softdtw_backward(Bp, gb, gamma, None, ws=ws)
        assert torch.equal(g_null, grad)
        wts.adam_step(Bp, grad, m, v, t, lr=lr)
    assert torch.equal(B, Bp)
    assert torch.equal(hist, torch.stack(hp))


def test_gamma_validation(wts):
    B, b = _case(9, 10, [10], 1)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    from paper_2404_12134_gb300._abi import WtsError
    with pytest.raises(WtsError):
        wts.softdtw_forward(torch.from_numpy(B).cuda(), gb, 0.0)


@pytest.mark.parametrize("G", [1, 3])
def test_checkpoint_mode_identical(wts, G):
    """dir_mode=1 keeps only the band hand-off rows; softdtw_backward
    recomputes R for G bands at a time: values and gradients identical."""
    B, b = _case(10, 1100, [900, 1300, 77], 1)       # several bands of 32 x rows-per-lane rows
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    w = torch.from_numpy((1.0 / b.lengths).astype(np.float32)).cuda()
    ws = wts.Workspace()
    v0 = wts.softdtw_forward(Bt, gb, 0.3, ws=ws)
    g0 = wts.softdtw_backward(Bt, gb, 0.3, w, ws=ws)
    opt = wts.options(dir_mode=1, ckpt_bands=G)
    ws1 = wts.Workspace()
    v1 = wts.softdtw_forward(Bt, gb, 0.3, opt, ws=ws1)
    g1 = wts.softdtw_backward(Bt, gb, 0.3, w, opt, ws=ws1)
    assert torch.equal(v0, v1) and torch.equal(g0, g1)
    s_ck = wts.workspace_size(wts._abi.OP_SOFTDTW, 1100, gb, opt)
    s_st = wts.workspace_size(wts._abi.OP_SOFTDTW, 1100, gb)
    assert s_ck <= s_st and (G > 1 or s_ck < s_st)


@pytest.mark.parametrize("M,d,cost", [(1100, 1, 0), (1024, 1, 0), (700, 3, 0), (520, 2, 1)])
def test_store_pairs_identical(wts, M, d, cost):
    """Column checkpoints with the longest pairs keeping R (store_pairs): the
    stored pairs' items run the backward that reads R, the others the fused
    one that recomputes it, in one launch.  Values and gradients equal, bit for bit,
    those with every R stored and with every pair checkpointed, also in batch
    order (keep_batch_order: the batch's first pairs keep R); with one
    channel and M a multiple of 8 (1024) the first launch is the one-channel
    backward without checked columns."""
    B, b = _case(70 + M, M, [900, 1300, 77, 1300, 31], d)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    w = torch.from_numpy((1.0 / b.lengths).astype(np.float32)).cuda()
    res = []
    for opt in (wts.options(cost_kind=cost), wts.options(dir_mode=1, cost_kind=cost),
                wts.options(dir_mode=1, cost_kind=cost, store_pairs=1),
                wts.options(dir_mode=1, cost_kind=cost, store_pairs=3),
                wts.options(dir_mode=1, cost_kind=cost, store_pairs=2, keep_batch_order=1),
                wts.options(dir_mode=1, cost_kind=cost, store_pairs=5)):
        ws = wts.Workspace()
        v = wts.softdtw_forward(Bt, gb, 0.1, opt, ws=ws)
        g = wts.softdtw_backward(Bt, gb, 0.1, w, opt, ws=ws)
        assert wts.read_status(ws.buf) == 0
        res.append((v, g))
    for v, g in res[1:]:
        assert torch.equal(v, res[0][0]) and torch.equal(g, res[0][1])


def test_adam_barycenter_store_pairs_identical(wts):
    """The library's Adam loop with two of five pairs keeping R beside column
    checkpoints reaches the barycenter of the stored mode, bit for bit."""
    b = synth.config_batch(2, scale=0.06, T=5)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M = 700
    B0 = wts.euclid_mean(gb, M)
    Bs, hs = wts.softdtw_barycenter(gb, M, 0.1, steps=5, lr=2e-2, init=B0)
    Bh, hh = wts.softdtw_barycenter(gb, M, 0.1, steps=5, lr=2e-2, init=B0,
                                    opts=wts.options(dir_mode=1, store_pairs=2))
    assert torch.equal(Bs, Bh) and torch.equal(hs, hh)


@pytest.mark.parametrize("dir_mode", [0, 1])
@pytest.mark.parametrize("M", [8, 256, 776, 1000, 1024])
def test_aligned_rows_backward_identical_to_checked(wts, M, dir_mode):
    """With one channel, no band and M a multiple of the 8 rows per lane, the
    backward runs no checked column: lanes past the matrix skip their columns
    and the seed e(M-1, N-1) = 1 enters as a diagonal successor of weight 1.
    Values and gradients equal, bit for bit, those of the checked backward,
    run here through a second channel of zeros (the same arithmetic in
    another kernel); with R stored and with column checkpoints."""
    B, b = _case(40 + M, M, [M, 1, 31, 300, M + 45, 2 * M + 3], 1)
    B2 = np.concatenate([B, np.zeros_like(B)], axis=1)
    c2 = [np.concatenate([b.cycle(k), np.zeros_like(b.cycle(k))], axis=1) for k in range(b.T)]
    b2 = synth.pack(c2)
    opt = wts.options(dir_mode=dir_mode, ckpt_bands=1 << 20) if dir_mode else None
    out = []
    for Bx, bx in ((B, b), (B2, b2)):
        gb = wts.Batch.from_numpy(bx.data, bx.offsets)
        Bt = torch.from_numpy(Bx).cuda()
        ws = wts.Workspace()
        v = wts.softdtw_forward(Bt, gb, 0.2, opt, ws=ws)
        g = wts.softdtw_backward(Bt, gb, 0.2, None, opt, ws=ws)
        assert wts.read_status(ws.buf) == 0
        out.append((v.cpu().numpy(), g.cpu().numpy()))
    (v1, g1), (v2, g2) = out
    assert (v1 == v2).all()
    assert (g1[:, 0] == g2[:, 0]).all() and (g2[:, 1] == 0).all()


def test_full_size_pair_value(wts):
    """The soft-DTW workload at full size (64 cycles of 8k-12k, M = 10,000,
    the benchmark's launch): two sampled pairs' values against the FP64
    oracle."""
    b = synth.config_batch(2)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M = synth.PROTO_LEN[2]
    B = wts.euclid_mean(gb, M)
    v = wts.softdtw_forward(B, gb, 1.0).cpu().numpy()
    Bh = B.cpu().numpy()
    for k in (0, 63):
        ref = oracle.softdtw(Bh, b.cycle(k), 1.0, "f64", want_grad=False)["value"]
        assert abs(v[k] - ref) <= VALUE_TOL * max(abs(ref), 1.0), (k, v[k], ref)


def test_lbfgs_barycenter_matches_oracle(wts):
    """Eq. 7 barycenter by L-BFGS with Table I's settings on a small batch: the
    library (objective and gradient from the GPU kernels, FP32) and the oracle
    (FP64) reach the same objective to 1e-3 relative; the objective never
    rises above the start's."""
    b = synth.config_batch(2, scale=0.008, T=5)          # 5 cycles of 64-96 samples
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M = 60
    B0 = wts.euclid_mean(gb, M)
    Bg, f, it, ev, why = wts.softdtw_barycenter_lbfgs(gb, M, 1.0, init=B0)
    assert why in ("ftol", "gtol", "max_iter", "max_fun") and it <= 40 and ev <= 200
    B0h = B0.cpu().numpy()
    w = (1.0 / b.lengths).astype(np.float32)
    _, f0, _ = oracle.softdtw_batch(B0h, b.data, b.offsets, 1.0, weights=w, prec="f64")
    Bo, fo, ito, evo, whyo = oracle.softdtw_barycenter_lbfgs(b.data, b.offsets, B0h, 1.0)
    _, fg, _ = oracle.softdtw_batch(Bg.cpu().numpy(), b.data, b.offsets, 1.0, weights=w, prec="f64")
    assert fg < f0 and fo < f0
    assert abs(fg - fo) <= 1e-3 * abs(fo), (fg, fo, it, ito)


@pytest.mark.parametrize("gamma", [1.0, 0.1])
@pytest.mark.parametrize("case,w", [((7, 300, [310, 200, 520], 1), 0.15), ((8, 520, [700, 260], 2), 0.3),
                                    ((9, 260, [260, 33], 3), 0.6)])
def test_banded_softdtw_value_and_gradient(wts, case, w, gamma):
    """Soft-DTW with Table I's Sakoe-Chiba band: values within the value bar
    of the FP64 oracle (restricted to in-band paths), gradients within the
    plain-FP32 bar; several row bands, M < N and M > N."""
    seed, M, lens, d = case
    B, b = _case(seed, M, lens, d)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B).cuda()
    o = wts.options(band=w)
    ws = wts.Workspace()
    v = wts.softdtw_forward(Bt, gb, gamma, o, ws=ws)
    wt = torch.from_numpy((1.0 / np.asarray(lens)).astype(np.float32)).cuda()
    g = wts.softdtw_backward(Bt, gb, gamma, wt, o, ws=ws)
    assert wts.read_status(ws.buf) == 0
    wd = 1.0 / np.asarray(lens, dtype=np.float64)
    vo, lo, go = oracle.softdtw_batch(B, b.data, b.offsets, gamma, weights=wd, band=w)
    vg = v.cpu().numpy().astype(np.float64)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(vg - vo) <= VALUE_TOL * np.maximum(np.abs(vo), 1.0)), np.abs(vg - vo).max()
    g32 = oracle.softdtw_batch(B, b.data, b.offsets, gamma, weights=wd.astype(np.float32), prec="f32", band=w)[2]
    bar = 2.0 * np.abs(g32.astype(np.float64) - go).max() / np.abs(go).max() + 1e-5
    assert np.abs(gg - go).max() / np.abs(go).max() <= bar
    # checkpointed R (recomputed per group of bands): the same gradient
    oc = wts.options(band=w, dir_mode=1, ckpt_bands=1)
    wts.softdtw_forward(Bt, gb, gamma, oc, ws=ws)
    gc = wts.softdtw_backward(Bt, gb, gamma, wt, oc, ws=ws)
    assert torch.equal(gc, g)


def test_banded_lbfgs_barycenter(wts):
    """Table I's full setting at small size: band 0.6, gamma 1, L-BFGS; the
    reached objective within 1e-3 of the oracle's (FP64, in-band paths)."""
    b = synth.config_batch(2, scale=0.008, T=5)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M = 60
    B0 = wts.euclid_mean(gb, M)
    Bg, f, it, ev, why = wts.softdtw_barycenter_lbfgs(gb, M, 1.0, init=B0, opts=wts.options(band=0.6))
    w = (1.0 / b.lengths).astype(np.float32)
    _, fg, _ = oracle.softdtw_batch(Bg.cpu().numpy(), b.data, b.offsets, 1.0, weights=w, prec="f64", band=0.6)
    Bo, fo, ito, evo, whyo = oracle.softdtw_barycenter_lbfgs(b.data, b.offsets, B0.cpu().numpy(), 1.0, band=0.6)
    assert abs(fg - fo) <= 1e-3 * abs(fo), (fg, fo)


def test_adam_barycenter_checkpoint_mode_identical(wts):
    """The library's Adam loop with R recomputed from column checkpoints
    (dir_mode = 1) reaches the same barycenter, bit for bit, as with R stored."""
    b = synth.config_batch(2, scale=0.06, T=5)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M = 700
    B0 = wts.euclid_mean(gb, M)
    Bs, hs = wts.softdtw_barycenter(gb, M, 0.1, steps=5, lr=2e-2, init=B0)
    Bc, hc = wts.softdtw_barycenter(gb, M, 0.1, steps=5, lr=2e-2, init=B0, opts=wts.options(dir_mode=1))
    assert torch.equal(Bs, Bc) and torch.equal(hs, hc)


def test_lbfgs_barycenter_reports_nonfinite_sample(wts):
    """A NaN sample stops the L-BFGS driver at its first evaluation with
    WTS_EINVAL (the device-side input scan), not with a wrong objective."""
    from paper_2404_12134_gb300._abi import WTS_EINVAL, WtsError
    b = synth.config_batch(2, scale=0.03, T=4)
    data = b.data.copy()
    data[17, 0] = np.nan
    gb = wts.Batch.from_numpy(data, b.offsets)
    with pytest.raises(WtsError) as ei:
        wts.softdtw_barycenter_lbfgs(gb, 200, 0.1, init=torch.zeros((200, 1), device="cuda"))
    assert ei.value.code == WTS_EINVAL


def test_lbfgs_first_step_matches_oracle(wts):
    """One L-BFGS iteration (max_iter = 1) from the same start: the step the
    library takes (GPU objective and gradient in FP32, the driver in double on
    the host) equals the oracle's (FP64) within the gradient's bar: twice a
    plain FP32 evaluation's error plus 1e-5, relative to the step's size (a
    first iteration is steepest descent, x1 = x0 - t g, with the same
    backtracking on both sides)."""
    b = synth.config_batch(2, scale=0.008, T=5)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    M, gamma = 60, 1.0
    B0 = wts.euclid_mean(gb, M)
    B0h = B0.cpu().numpy()
    Bg, f, it, ev, why = wts.softdtw_barycenter_lbfgs(gb, M, gamma, init=B0, params=wts.lbfgs_params(max_iter=1))
    Bo, fo, ito, evo, whyo = oracle.softdtw_barycenter_lbfgs(b.data, b.offsets, B0h, gamma, max_iter=1)
    assert it == ito == 1 and ev == evo
    w = (1.0 / b.lengths).astype(np.float32)
    _, _, go = oracle.softdtw_batch(B0h, b.data, b.offsets, gamma, weights=w.astype(np.float64))
    bar = _grad_bar(B0h, b, gamma, w.astype(np.float64), go)
    dg = Bg.cpu().numpy().astype(np.float64) - B0h
    do = np.asarray(Bo, dtype=np.float64).reshape(B0h.shape) - B0h
    assert np.abs(dg - do).max() <= 2.0 * bar * np.abs(do).max() + 1e-7, (np.abs(dg - do).max(), np.abs(do).max())

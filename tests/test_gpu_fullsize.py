"""Full-size parity through the C ABI at the benchmark workloads' own sizes,
with the error against the FP64 oracle stated for every result.

* One DBA iteration on 16 full-length cycles of the batched-DBA workload
  (M = 25,000, d = 6, the benchmark's launch shape, a 13-round segmented
  walk): prototype, counts, per-cycle costs and the FP64 cost sum bit-exact
  against the FP32 mirror; against FP64: the prototype's and the costs'
  relative errors and the number of path cells where the FP32 path leaves
  the FP64 path.
* One Soft-DTW pair of the barycenter workload (M = 10,000, N ~ 10k) at the
  workload's three gammas: value within 1e-5 of FP64 (relative to
  max(|v|, 1)) or within twice a plain FP32 evaluation's error, whichever is
  larger (a path of ~19k cells rounds r once per cell: a plain FP32
  evaluation itself is ~1e-5 off at this size), and the Eq. 7 gradient within
  twice a plain FP32 evaluation's error plus 1e-5 (relative to the largest
  component).
* One pair of the very-long workload (M = 110,000, N ~ 108k, 3 channels) with
  checkpointed codes (16-band groups, as benchmarked): cost, |pi| and the
  path bit-exact against the FP32 mirror (the mirror keeps a 1-byte choice
  per cell: 12 GB of host memory; with less memory available the pair is cut
  to the largest size that fits, and the test says which).
* Checkpointed Soft-DTW with 64-band groups (as benchmarked) at the largest
  size whose FP64 R, Delta and E fit in host memory comfortably (M = N ~
  20,000, two groups): value and gradient against FP64.

Every FP64 error is printed on a line starting "FP64-ERROR" (run with -s).
"""
import os
from concurrent.futures import ThreadPoolExecutor

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


def _mem_available_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


def _path_cells_differing(jlo_a, jhi_a, jlo_b, jhi_b) -> int:
    """Cells in exactly one of two monotone paths given by per-row column ranges."""
    la = jhi_a.astype(np.int64) - jlo_a + 1
    lb = jhi_b.astype(np.int64) - jlo_b + 1
    ov = np.maximum(0, np.minimum(jhi_a, jhi_b).astype(np.int64) - np.maximum(jlo_a, jlo_b) + 1)
    return int((la + lb - 2 * ov).sum())


def test_batched_dba_iteration_16_full_length_cycles(wts):
    b = synth.config_batch(1, T=16)
    M = 25000
    B0 = oracle.resample(b.cycle(0), M)
    gb = wts.Batch.from_numpy(b.data, b.offsets)
    Bt = torch.from_numpy(B0).cuda()
    opt = wts.options(rows_per_thread=16, warps_per_block=4)      # the benchmark's launch shape
    ws = wts.Workspace()
    Bn, cnt, cb, ck = wts.dba_iterate(Bt, gb, opt, ws=ws)
    _, plen, jlo, jhi = wts.dtw_align(Bt, gb, opt, ws=ws)
    assert wts.read_status(ws.buf) == 0
    Bo, cnt_o, cb_o, ck_o = oracle.dba_iterate(B0, b.data, b.offsets, "f32")
    assert (Bn.cpu().numpy() == Bo).all()
    assert (cnt.cpu().numpy() == cnt_o).all()
    assert float(cb) == cb_o
    assert (ck.cpu().numpy() == ck_o).all()
    # against FP64: the same iteration in double, and the FP64 paths.  Where
    # FP32 and FP64 choose the same path cells for every cycle, the averaging
    # adds the same samples in the same order in double, so the prototype row
    # is the FP64 one rounded to FP32, exactly; elsewhere a near-tie of two
    # path costs (closer than the FP32 rounding of r) was decided the other
    # way, and the row averages other samples: that error is stated.
    B64, cnt64, cb64, ck64 = oracle.dba_iterate(B0.astype(np.float64), b.data, b.offsets, "f64")
    jl, jh = jlo.cpu().numpy(), jhi.cpu().numpy()
    threads = max(1, min(os.cpu_count() or 1, 16, int(_mem_available_gb() // 1.5)))

    def one(k):
        r = oracle.dtw(B0, b.cycle(k), "f64", path=False)
        return r["jlo"], r["jhi"]

    with ThreadPoolExecutor(threads) as ex:
        p64 = list(ex.map(one, range(b.T)))
    diff = [_path_cells_differing(jl[k], jh[k], *p64[k]) for k in range(b.T)]
    same_rows = np.ones(M, dtype=bool)
    for k in range(b.T):
        same_rows &= (jl[k] == p64[k][0]) & (jh[k] == p64[k][1])
    Bg = Bn.cpu().numpy()
    assert (Bg[same_rows] == B64[same_rows].astype(np.float32)).all()
    e = np.abs(Bg.astype(np.float64) - B64)
    cost_rel = np.abs(ck.cpu().numpy().astype(np.float64) - ck64) / np.abs(ck64)
    print(f"FP64-ERROR batched DBA, 16 x ~24.5k x 6 ch, M=25000, one iteration: path cells differing "
          f"{sum(diff)} of {int(plen.cpu().numpy().sum())} (in {sum(1 for x in diff if x)} of 16 pairs); "
          f"prototype rows with every range equal {int(same_rows.sum())} of {M}, there equal to FP64 rounded "
          f"to FP32; elsewhere max abs {e[~same_rows].max() if (~same_rows).any() else 0.0:.3e} "
          f"(max|B| {np.abs(B64).max():.3g}); per-cycle cost max rel {cost_rel.max():.3e}; cost sum rel "
          f"{abs(float(cb) - cb64) / cb64:.3e}")
    assert cost_rel.max() <= 1e-5 and abs(float(cb) - cb64) <= 1e-5 * cb64


@pytest.mark.parametrize("gamma", [1.0, 0.1, 0.01])
def test_softdtw_pair_full_size_value_and_gradient(wts, gamma):
    b = synth.config_batch(2, T=2)
    M = 10000
    B = oracle.resample(b.cycle(1), M)
    y = b.cycle(0)
    one = synth.pack([y])
    gb = wts.Batch.from_numpy(one.data, one.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    v = wts.softdtw_forward(Bt, gb, gamma, ws=ws)
    g = wts.softdtw_backward(Bt, gb, gamma, None, ws=ws)            # Eq. 7 weight 1 / N
    assert wts.read_status(ws.buf) == 0
    w = np.array([1.0 / len(y)], dtype=np.float32)
    vo, _, go = oracle.softdtw_batch(B, one.data, one.offsets, gamma, weights=w.astype(np.float64))
    v32, _, g32 = oracle.softdtw_batch(B, one.data, one.offsets, gamma, weights=w, prec="f32")
    vg = float(v.cpu().numpy()[0])
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.abs(go).max()
    gerr = np.abs(gg - go).max() / scale
    g32err = np.abs(g32.astype(np.float64) - go).max() / scale
    vden = max(abs(float(vo[0])), 1.0)
    verr = abs(vg - float(vo[0])) / vden
    v32err = abs(float(v32[0]) - float(vo[0])) / vden
    print(f"FP64-ERROR soft-DTW pair {M} x {len(y)}, gamma={gamma}: value rel {verr:.3e} (plain FP32 "
          f"evaluation: {v32err:.3e}); gradient max / max|g| {gerr:.3e} (plain FP32 evaluation: {g32err:.3e})")
    assert verr <= max(1e-5, 2.0 * v32err)
    assert gerr <= 2.0 * g32err + 1e-5


def test_very_long_pair_checkpointed_paths_bit_exact(wts):
    b = synth.config_batch(4, T=2)
    M = 110000
    y = b.cycle(1)
    need_gb = 1.3 * M * len(y) / 1e9 + 2.0
    avail = _mem_available_gb()
    if avail and avail < need_gb:
        s = np.sqrt(max(avail - 2.0, 1.0) / 1.3 * 1e9 / (M * len(y)))
        M, y = int(M * s), y[: int(len(y) * s)]
    B = oracle.resample(b.cycle(0), M)
    one = synth.pack([y])
    gb = wts.Batch.from_numpy(one.data, one.offsets)
    Bt = torch.from_numpy(B).cuda()
    ws = wts.Workspace()
    ck = wts.dtw_align(Bt, gb, wts.options(dir_mode=1, ckpt_bands=16), ws=ws)
    assert wts.read_status(ws.buf) == 0
    st = wts.dtw_align(Bt, gb, ws=ws)
    for a, c in zip(ck, st):
        assert torch.equal(a, c)
    cost, plen, jlo, jhi = (t.cpu().numpy() for t in ck)
    r = oracle.dtw(B, y, "f32", path=False)
    print(f"very long pair {M} x {len(y)} x 3 ch (checkpointed codes, 16-band groups); "
          f"host memory available {avail:.0f} GB")
    assert float(cost[0]) == float(r["cost"]) and int(plen[0]) == r["plen"]
    assert (jlo[0] == r["jlo"]).all() and (jhi[0] == r["jhi"]).all()


def test_checkpointed_softdtw_largest_oracle_size(wts):
    b = synth.config_batch(4, scale=0.18, T=2)
    M = 20000
    B = oracle.resample(b.cycle(0), M)
    y = b.cycle(1)
    one = synth.pack([y])
    gb = wts.Batch.from_numpy(one.data, one.offsets)
    Bt = torch.from_numpy(B).cuda()
    gamma = 0.1
    ws = wts.Workspace()
    opt = wts.options(dir_mode=1, ckpt_bands=64)
    v = wts.softdtw_forward(Bt, gb, gamma, opt, ws=ws)
    g = wts.softdtw_backward(Bt, gb, gamma, None, opt, ws=ws)
    assert wts.read_status(ws.buf) == 0
    w = np.array([1.0 / len(y)], dtype=np.float32)
    vo, _, go = oracle.softdtw_batch(B, one.data, one.offsets, gamma, weights=w.astype(np.float64))
    v32, _, g32 = oracle.softdtw_batch(B, one.data, one.offsets, gamma, weights=w, prec="f32")
    scale = np.abs(go).max()
    gerr = np.abs(g.cpu().numpy().astype(np.float64) - go).max() / scale
    g32err = np.abs(g32.astype(np.float64) - go).max() / scale
    vden = max(abs(float(vo[0])), 1.0)
    verr = abs(float(v.cpu().numpy()[0]) - float(vo[0])) / vden
    v32err = abs(float(v32[0]) - float(vo[0])) / vden
    print(f"FP64-ERROR checkpointed soft-DTW pair {M} x {len(y)} x 3 ch, gamma={gamma}, 64-band groups: "
          f"value rel {verr:.3e} (plain FP32: {v32err:.3e}); gradient max / max|g| {gerr:.3e} "
          f"(plain FP32: {g32err:.3e})")
    assert verr <= max(1e-5, 2.0 * v32err)
    assert gerr <= 2.0 * g32err + 1e-5

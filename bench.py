#!/usr/bin/env python
"""Benchmark of the WETSAND alignment hot path on one GB300 (or N replicas).

Workload (the batched-DBA configuration): 200 synthetic cycles, 6 channels,
FP32, pre-gap lengths U(20k, 30k) with 2 % gaps removed, 10 % anomalous,
prototype length M = 25,000 (initialised, untimed, from the medoid of a seeded
16-cycle subset resampled to M).  One step = one DBA iteration: the DTW
wavefront with 2-bit predecessor codes over all 200 pairs, the backtrack and
the averaging.  The metric is DTW cells per second (GCUPS, M * sum N_k cells
per step) and seconds per DBA iteration; soft-DTW forward + backward GCUPS
and anomaly-score GCUPS are reported beside it.

--impl reference times the CPU oracle (the plain C implementation the tests
check against) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2404_12134_gb300 import synth  # noqa: E402

M_PROTO = synth.PROTO_LEN[1]
WORKLOAD = ("batched DBA: 200 cycles x 6 ch FP32, pre-gap N ~ U(20k,30k), 2% gaps, "
            "10% anomalous, M=25000, one DBA iteration per step")
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per cell of the code-writing wavefront, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the same
# kernel build on 36 cycles of this workload: (0.16208 + 5.64213)e9 bytes /
# 2.2029e10 cells.  Traffic grows in proportion to the cells (codes +
# hand-off rows).
WAVEFRONT_DIRS_DRAM_BYTES_PER_CELL = (0.16208 + 5.64213) * 1e9 / 2.2029e10
# DRAM bytes (read + write) per cell of soft-DTW forward + backward, from one
# ncu capture of both kernels (the same build) on the soft-DTW workload with
# its cycles cut to an eighth (64 pairs, the benchmark's occupancy):
# (0.01512 + 3.26850 + 3.36838 + 0.05043)e9 bytes / 7.9029e8 cells (stored R plus
# hand-off rows, in proportion to cells; the skew margin, 2.5 % of a band at
# that length, is 0.3 % at full length).
SOFT_FWD_BWD_DRAM_BYTES_PER_CELL = (0.01512 + 3.26850 + 3.36838 + 0.05043) * 1e9 / 7.9029e8
# Warp instructions per cell of the checkpointed soft-DTW passes (column
# checkpoints, recompute fused into the backward), from one ncu capture
# (smsp__inst_executed.sum) of the same build on the very-long workload's
# 8 pairs cut to a quarter (5.842e9 cells): forward 4.9229e9, backward
# 1.20786e10.  Both passes are bound by the issue rate (one warp instruction
# per scheduler per cycle), not by a pipe or by DRAM.
SOFT_CKPT_FWD_INSTR_PER_CELL = 4.9229e9 / 5.842045e9
SOFT_CKPT_BWD_INSTR_PER_CELL = 1.20786e10 / 5.842045e9


def softckpt_roofline(cells: int, fwd_ms: float, bwd_ms: float, sms: int, ex2: float | None, lg2: float | None):
    """Issue-rate roofline of the checkpointed soft-DTW passes (and their MUFU
    fraction when the measured ex2 / lg2 rates are given)."""
    peak = sms * 4 * 2.070e9                         # warp instructions per second
    out = {}
    for name, ms, ipc, mufu in (("fwd", fwd_ms, SOFT_CKPT_FWD_INSTR_PER_CELL, (2, 1)),
                                ("bwd", bwd_ms, SOFT_CKPT_BWD_INSTR_PER_CELL, (5, 1))):
        t = ms * 1e-3
        r = {"bound": "issue", "achieved": cells * ipc / t, "peak": peak, "unit": "warp-instructions/s",
             "frac": cells * ipc / t / peak, "instructions_per_cell": ipc,
             "peak_note": f"{sms} SMs x 4 schedulers x 2070 MHz; instructions per cell from one ncu capture"}
        if ex2 and lg2:
            r["mufu_frac"] = cells * (mufu[0] / ex2 + mufu[1] / lg2) / t
        out[name] = r
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wetsand", choices=["wetsand", "reference"])
    ap.add_argument("--T", type=int, default=200, help="cycles (default: the full workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the score / soft-DTW side metrics")
    ap.add_argument("--soft-ckpt", action="store_true",
                    help="soft leg in checkpoint mode (R recomputed in the backward; for profiling)")
    ap.add_argument("--leg", default="all",
                    choices=["all", "dba", "soft", "score", "long", "bary", "table", "segment", "softckpt", "small"],
                    help="only that leg (soft: --T cycles of its workload, lengths times --scale; softckpt: the "
                         "very-long workload's checkpointed soft-DTW on --T pairs, lengths times --scale); "
                         "for profiling")
    ap.add_argument("--scale", type=float, default=1.0, help="length scale of the soft / softckpt legs' cycles")
    ap.add_argument("--store-pairs", type=int, default=0, help="softckpt leg: pairs that keep R beside the checkpoints")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's value (whole-job time is set by the last rank to
    finish); identity on one rank."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(T: int):
    b = synth.config_batch(1, T=T)
    rng = np.random.default_rng(synth.SEED_BASE + 77)
    subset = np.sort(rng.choice(b.T, size=min(16, b.T), replace=False))
    return b, subset


# --- clocks ---------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.lines = []
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --- CPU oracle timing (baseline and reference arm) ---------------------------

def oracle_dba_sample(b, B, n_cycles: int, prec: str = "f64"):
    """Time one oracle DBA iteration on the first n_cycles cycles; returns (GCUPS, seconds, cells)."""
    import oracle
    sub = b.subset(np.arange(n_cycles))
    cells = int(B.shape[0]) * int(sub.lengths.sum())
    t0 = time.perf_counter()
    oracle.dba_iterate(B.astype(np.float64) if prec == "f64" else B, sub.data, sub.offsets, prec)
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, dt, cells


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    ncores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
    import oracle
    oracle.build()
    b, subset = make_workload(args.T)
    B = synth.clean_prototype(b, M_PROTO)      # the oracle's step cost does not depend on B's values
    n = min(ncores, b.T)
    for _ in range(args.warmup):
        oracle_dba_sample(b, B, n)
    tot_t, tot_c = 0.0, 0
    for _ in range(args.steps):
        g, dt, cells = oracle_dba_sample(b, B, n)
        tot_t += dt; tot_c += cells
    val = tot_c / tot_t / 1e9
    sample = f"{n} of {b.T} cycles per step (one oracle DBA iteration, FP64, M={M_PROTO}), {ncores} OpenMP threads"
    print(json.dumps({
        "impl": "reference", "metric": "dtw_gcups_dba_iteration", "value": val, "unit": "GCUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": b.T, "d": b.d, "M": M_PROTO},
        "cpu_baseline": {"value": val, "unit": "GCUPS", "cores": ncores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# --- GPU arm ----------------------------------------------------------------------

def hbm_peak_gbs() -> float:
    """Measured HBM copy bandwidth (generated file), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def softdtw_leg(api, torch, dev, st, barrier, gamma: float = 1.0, T: int | None = None, ckpt: bool = False,
                band: float = 0.0, per_pair: bool = False, peaks: dict | None = None, scale: float = 1.0,
                wpb: int = 0):
    """Soft-DTW forward + backward on the single-channel barycenter workload:
    64 cycles, pre-gap N ~ U(8k, 12k), M = 10,000 (R stored: ~26 GB), the
    Eq. 7 weights 1 / N_k (the library's default);
    band > 0: with the Sakoe-Chiba band (GCUPS then also over the cells in
    the band); per_pair: also the plain form, one forward + backward call per
    cycle; peaks (measured ex2 / lg2 rates): a roofline for each kernel."""
    sb = synth.config_batch(2, T=T, scale=scale)
    M = synth.PROTO_LEN[2]
    gb = api.Batch.from_numpy(sb.data, sb.offsets, device=dev)
    B = api.euclid_mean(gb, M)
    w = None
    ws = api.Workspace(dev)
    grad = torch.empty_like(B)
    opt = api.options(dir_mode=1, ckpt_bands=1 << 20, band=band, warps_per_block=wpb) if ckpt else \
        api.options(band=band, warps_per_block=wpb)
    for _ in range(2):
        api.softdtw_forward(B, gb, gamma, opt, ws=ws)
        api.softdtw_backward(B, gb, gamma, w, opt, ws=ws, grad_B=grad)
    barrier()
    api.profile_read("")
    api.profile_enable(True)
    reps = 3
    for _ in range(reps):
        vals = api.softdtw_forward(B, gb, gamma, opt, ws=ws)
        api.softdtw_backward(B, gb, gamma, w, opt, ws=ws, grad_B=grad)
    barrier()
    api.profile_enable(False)
    f_ms, _ = api.profile_read("softdtw_fwd")
    b_ms, _ = api.profile_read("softdtw_bwd")
    g_ms, _ = api.profile_read("softdtw_grad")
    api.profile_read("")
    cells = M * int(sb.lengths.sum())
    fwd, bwd = f_ms / reps, (b_ms + g_ms) / reps
    res = {"workload": "64 cycles x 1 ch FP32, pre-gap N ~ U(8k,12k), 2% gaps, M=10000, Euclidean-mean init",
           "gamma": gamma, "cells": cells, "fwd_ms": fwd, "bwd_ms": bwd,
           "fwd_bwd_gcups": cells / ((fwd + bwd) * 1e-3) / 1e9,
           "fwd_gcups": cells / (fwd * 1e-3) / 1e9, "bwd_gcups": cells / (bwd * 1e-3) / 1e9,
           "workspace_gb": ws.buf.numel() / 1e9, "device_status": api.read_status(ws.buf),
           "loss": float((vals.double().cpu().numpy() * (1.0 / sb.lengths).astype(np.float32)).sum())}
    if band:
        inb = band_cells(M, sb.lengths, band)
        res.update(band=band, cells_in_band=inb, fwd_bwd_gcups_in_band=inb / ((fwd + bwd) * 1e-3) / 1e9)
    if peaks and not band and not ckpt:
        # per kernel: the MUFU bound (forward 2 ex2 + 1 lg2 per cell, backward
        # 3 ex2) and the HBM bound of the stored R (4 B written per cell
        # forward, 4 B read backward); the larger one is the kernel's roofline
        hbm = hbm_peak_gbs() * 1e9
        for name, ms, mufu_s in (("fwd", fwd, cells * (2 / peaks["ex2"] + 1 / peaks["lg2"])),
                                 ("bwd", bwd, cells * 3 / peaks["ex2"])):
            hbm_s = cells * 4 / hbm
            t = ms * 1e-3
            if hbm_s >= mufu_s:
                res[f"roofline_{name}"] = {"bound": "hbm", "achieved": cells * 4 / t / 1e9, "peak": hbm / 1e9,
                                           "unit": "GB/s", "frac": hbm_s / t, "mufu_frac": mufu_s / t}
            else:
                res[f"roofline_{name}"] = {"bound": "mufu", "frac": mufu_s / t, "hbm_frac": hbm_s / t}
    if per_pair:
        # the plain form: one forward + backward call per cycle, in turn
        ws1 = api.Workspace(dev)
        singles = []
        for k in range(sb.T):
            o0, o1 = int(sb.offsets[k]), int(sb.offsets[k + 1])
            singles.append(api.Batch(gb.data[o0:o1], torch.tensor([0, o1 - o0], device=dev),
                                     np.array([0, o1 - o0], dtype=np.int64)))
        api.softdtw_forward(B, singles[0], gamma, None, ws=ws1)
        api.softdtw_backward(B, singles[0], gamma, None, None, ws=ws1, grad_B=grad)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for one in singles:
            api.softdtw_forward(B, one, gamma, None, ws=ws1)
            api.softdtw_backward(B, one, gamma, None, None, ws=ws1, grad_B=grad)
        e1.record()
        barrier()
        pp = e0.elapsed_time(e1)
        res["per_pair_launch_ms"] = pp
        res["per_pair_launch_fwd_bwd_gcups"] = cells / (pp * 1e-3) / 1e9
        del ws1
    del ws, gb
    return res


def scoring_leg(api, torch, dev, barrier, T: int | None = None, per_pair: bool = True):
    """Uneven scoring: 1,000 cycles x 3 ch, pre-gap lengths log-normal (median
    15k, sigma 0.6) clipped to 2k-60k, 5 % anomalous (drift / skipped segment /
    3x slowdown), scored against the clean base sampled at M = 20,000.  One
    persistent launch (autotuned options, captured in a CUDA graph) against one
    launch per pair."""
    from paper_2404_12134_gb300 import _abi
    b = synth.config_batch(3, T=T)
    M = synth.PROTO_LEN[3]
    B = torch.from_numpy(synth.clean_prototype(b, M)).to(dev)
    gb = api.Batch.from_numpy(b.data, b.offsets, device=dev)
    cells = M * int(b.lengths.sum())
    ws = api.Workspace(dev)
    opts, tune_ms = api.autotune(_abi.OP_ANOMALY_SCORE, B, gb, ws)
    g, (score, cost, plen) = api.capture(lambda: api.anomaly_score(B, gb, opts, ws=ws))
    g.replay()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    barrier()
    batched_ms = e0.elapsed_time(e1) / reps
    res = {"workload": "1000 cycles x 3 ch FP32, pre-gap N ~ lognormal(15k, 0.6) clipped 2k-60k, 5% anomalous, "
                       "M=20000 clean prototype",
           "T": b.T, "cells": cells, "options": {"rows_per_thread": opts.rows_per_thread,
                                                  "warps_per_block": opts.warps_per_block,
                                                  "form": "codes + walk" if opts.score_via_codes
                                                  else "count inside the DP"},
           "batched_graph_ms": batched_ms, "batched_gcups": cells / (batched_ms * 1e-3) / 1e9,
           "autotune_best_wavefront_ms": tune_ms}
    # the two detection thresholds of Sec. 5.3 on the scores, against the
    # injected anomalies (library host functions; not part of the timed path)
    sc = score.cpu().numpy()
    two_sigma, boxplot = api.thresholds(sc)
    res["boxplot_threshold"] = dict(api.f2_score(sc, b.labels, boxplot), threshold=boxplot)
    res["two_sigma_threshold"] = dict(api.f2_score(sc, b.labels, two_sigma), threshold=two_sigma)
    if per_pair:
        singles = []
        for k in range(b.T):
            o0, o1 = int(b.offsets[k]), int(b.offsets[k + 1])
            singles.append(api.Batch(gb.data[o0:o1], torch.tensor([0, o1 - o0], device=dev),
                                     np.array([0, o1 - o0], dtype=np.int64)))
        ws1 = api.Workspace(dev)
        api.anomaly_score(B, singles[0], ws=ws1)
        barrier()
        e0.record()
        for one in singles:
            api.anomaly_score(B, one, ws=ws1)
        e1.record()
        barrier()
        pp_ms = e0.elapsed_time(e1)
        g1, _ = api.capture(lambda: [api.anomaly_score(B, one, ws=ws1) for one in singles])
        g1.replay()
        barrier()
        e0.record()
        g1.replay()
        e1.record()
        barrier()
        ppg_ms = e0.elapsed_time(e1)
        res.update({"per_pair_eager_ms": pp_ms, "per_pair_eager_gcups": cells / (pp_ms * 1e-3) / 1e9,
                    "per_pair_graph_ms": ppg_ms, "per_pair_graph_gcups": cells / (ppg_ms * 1e-3) / 1e9,
                    "speedup_vs_per_pair_eager": pp_ms / batched_ms})
        del g1, ws1
    del g, ws
    torch.cuda.empty_cache()
    return res


def long_leg(api, torch, dev, barrier, iters: int = 2, cpu_sample: bool = True, ex2: float | None = None,
             lg2: float | None = None):
    """Very long cycles: 32 cycles x 3 ch, pre-gap N ~ U(100k, 120k), M =
    110,000 (medoid of a seeded 8-cycle subset, resampled; untimed).  DBA with
    every code stored (~95 GB) against checkpoint mode (band rows kept, codes
    recomputed 16 bands at a time), and soft-DTW forward + backward on 8 of the
    pairs with checkpointing (stored R would take ~390 GB), first, while the
    device memory is least fragmented."""
    import gc
    api.release_default_workspaces()     # earlier legs' default workspaces: the soft-DTW runs size by free memory
    gc.collect()
    torch.cuda.empty_cache()
    b = synth.config_batch(4)
    M = synth.PROTO_LEN[4]
    gb = api.Batch.from_numpy(b.data, b.offsets, device=dev)
    cells = M * int(b.lengths.sum())
    sub = b.subset(np.arange(8))
    gsub = api.Batch.from_numpy(sub.data, sub.offsets, device=dev)
    idx, _ = api.medoid(api.pairwise_dtw(gsub, ws=api.Workspace(dev)))
    k = int(idx)
    B0 = api.resample(gsub.data[int(sub.offsets[k]):int(sub.offsets[k + 1])], M)
    res = {"workload": "32 cycles x 3 ch FP32, pre-gap N ~ U(100k,120k), 2% gaps, M=110000", "cells_per_iter": cells}
    # soft-DTW forward + backward, 8 pairs, column checkpoints (stored R would
    # take ~390 GB); then with as many pairs keeping R as the free memory holds
    gamma = 0.1
    scells = M * int(sub.lengths.sum())
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_ms, b_ms, wgb, st, v_ck, g_ck = soft_fwd_bwd(api, torch, dev, barrier, B0, gsub, gamma, api.options(dir_mode=1))
    res["softdtw_checkpoint"] = {"pairs": 8, "gamma": gamma, "checkpoints": "every 16 steps per band", "cells": scells,
                                 "fwd_ms": f_ms, "bwd_incl_recompute_ms": b_ms,
                                 "fwd_bwd_gcups": scells / ((f_ms + b_ms) * 1e-3) / 1e9,
                                 "workspace_gb": wgb, "device_status": st,
                                 "roofline": softckpt_roofline(scells, f_ms, b_ms, sms, ex2, lg2)}
    # the most pairs whose R fits, and two fewer (the fewer pairs recompute,
    # the faster the backward, as long as the checkpointed pairs' items and
    # the stored pairs' items fill the resident warps)
    S, _ = api.store_pairs_for_memory(M, gsub)
    free_gb = torch.cuda.mem_get_info(dev)[0] / 1e9
    held_gb = (torch.cuda.memory_allocated(dev) / 1e9, torch.cuda.memory_reserved(dev) / 1e9)
    runs = []
    for s in range(S, max(0, S - 3), -1):
        try:
            f_ms, b_ms, wgb, st, v_h, g_h = soft_fwd_bwd(api, torch, dev, barrier, B0, gsub, gamma,
                                                         api.options(dir_mode=1, store_pairs=s))
        except torch.cuda.OutOfMemoryError:
            torch.cuda.empty_cache()
            runs.append({"store_pairs": s, "skipped": "the workspace did not fit"})
            continue
        runs.append({"store_pairs": s, "fwd_ms": f_ms, "bwd_incl_recompute_ms": b_ms,
                     "fwd_bwd_gcups": scells / ((f_ms + b_ms) * 1e-3) / 1e9, "workspace_gb": wgb,
                     "device_status": st,
                     "identical_to_checkpointed": bool(torch.equal(v_h, v_ck) and torch.equal(g_h, g_ck))})
        del v_h, g_h
    done = [r for r in runs if "fwd_bwd_gcups" in r]
    if done:
        best = max(done, key=lambda r: r["fwd_bwd_gcups"])
        res["softdtw_checkpoint"]["store_pairs"] = dict(
            best, note="the longest pairs keep R in HBM (store_pairs), the others column checkpoints; "
                       "best of the runs listed", runs=runs, free_gb_before=free_gb,
            torch_allocated_reserved_gb=held_gb)
    del v_ck, g_ck
    torch.cuda.empty_cache()
    outs = {}
    from paper_2404_12134_gb300 import _abi
    ws = api.Workspace(dev)
    tuned, _ = api.autotune(_abi.OP_DBA_ITERATE, B0, gb, ws)
    res["options"] = {"rows_per_thread": tuned.rows_per_thread, "warps_per_block": tuned.warps_per_block}
    for name, mode in (("stored", 0), ("checkpoint", 1)):
        opt = api.options(rows_per_thread=tuned.rows_per_thread, warps_per_block=tuned.warps_per_block,
                          dir_mode=mode, ckpt_bands=16)
        if ws is None:
            ws = api.Workspace(dev)
        B = B0.clone()
        Bn, cnt, cb, _ = api.dba_iterate(B, gb, opt, ws=ws)          # warm-up
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            Bn, cnt, cb, _ = api.dba_iterate(B, gb, opt, ws=ws)
            B, Bn = Bn, B
        e1.record()
        barrier()
        ms = e0.elapsed_time(e1) / iters
        outs[name] = B.clone()
        res[name] = {"s_per_dba_iter": ms * 1e-3, "gcups": cells / (ms * 1e-3) / 1e9,
                     "workspace_gb": api.workspace_size(_abi.OP_DBA_ITERATE, M, gb, opt) / 1e9,
                     "device_status": api.read_status(ws.buf)}
        ws = None
        torch.cuda.empty_cache()
    res["checkpoint_prototype_identical"] = bool(torch.equal(outs["stored"], outs["checkpoint"]))
    if cpu_sample:
        # the oracle (FP64) on a bounded sample: a full pair keeps a 1-byte
        # choice per cell (12 GB of host memory) and takes about a minute on
        # one core, so 16 cycles are cut to their first 2,000 samples and
        # aligned against the whole 110,000-row prototype, one per thread
        import oracle
        ncores = os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
        n = min(16, ncores, b.T)
        cut = [b.cycle(k)[:2000] for k in range(n)]
        sb = synth.pack(cut)
        Bh = synth.clean_prototype(b, M)       # the oracle's inputs come from the generator only
        t0 = time.perf_counter()
        oracle.score(Bh, sb.data, sb.offsets, "f64")
        dt = time.perf_counter() - t0
        c = M * int(sb.lengths.sum())
        res["cpu_oracle_subset"] = {"sample": f"{n} cycles cut to their first 2,000 samples against the full "
                                              f"{M}-row prototype, DTW + |pi| (FP64), one cycle per thread",
                                    "s": dt, "gcups": c / dt / 1e9, "threads": n, "cells": c}
    return res


def soft_fwd_bwd(api, torch, dev, barrier, B0, gb, gamma, opt):
    """One warm-up and one timed soft-DTW forward + backward (Eq. 7's default
    weights 1 / N_k); returns (fwd ms, bwd ms, workspace GB, status, values,
    gradient).  The workspace is freed before returning."""
    ws = api.Workspace(dev)
    api.softdtw_forward(B0, gb, gamma, opt, ws=ws)
    api.softdtw_backward(B0, gb, gamma, None, opt, ws=ws)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record()
    v = api.softdtw_forward(B0, gb, gamma, opt, ws=ws)
    e1.record()
    g = api.softdtw_backward(B0, gb, gamma, None, opt, ws=ws)
    e2.record()
    barrier()
    out = (e0.elapsed_time(e1), e1.elapsed_time(e2), ws.buf.numel() / 1e9, api.read_status(ws.buf), v, g)
    del ws
    torch.cuda.empty_cache()
    return out


def softckpt_leg(api, torch, dev, barrier, T: int = 8, scale: float = 1.0, gamma: float = 0.1, wpb: int = 0,
                 store_pairs: int = 0):
    """The very-long workload's checkpointed soft-DTW alone: T pairs of its
    cycles (lengths times scale) against a prototype of 110,000 x scale
    samples (the clean base; untimed), forward + backward with recomputation,
    one warm-up then one timed pass."""
    b = synth.config_batch(4, T=T, scale=scale)
    M = int(round(synth.PROTO_LEN[4] * scale))
    gb = api.Batch.from_numpy(b.data, b.offsets, device=dev)
    B0 = torch.from_numpy(synth.clean_prototype(b, M)).to(dev)
    opt = api.options(dir_mode=1, warps_per_block=wpb, store_pairs=store_pairs)
    f_ms, b_ms, wgb, st, _, _ = soft_fwd_bwd(api, torch, dev, barrier, B0, gb, gamma, opt)
    cells = M * int(b.lengths.sum())
    res = {"pairs": b.T, "M": M, "gamma": gamma, "cells": cells, "store_pairs": store_pairs, "fwd_ms": f_ms,
           "bwd_incl_recompute_ms": b_ms, "fwd_bwd_gcups": cells / ((f_ms + b_ms) * 1e-3) / 1e9,
           "workspace_gb": wgb, "device_status": st,
           "roofline": softckpt_roofline(cells, f_ms, b_ms, torch.cuda.get_device_properties(dev).multi_processor_count,
                                         None, None)}
    torch.cuda.empty_cache()
    return res


def bary_leg(api, torch, dev, barrier, gammas=(1.0, 0.1, 0.01), steps: int = 50, dba_iters: int = 10,
             lr: float = 5e-2):
    """Barycenters of the single-channel workload (64 cycles, M = 10,000): the
    Euclidean mean of the resampled cycles (Table I's initialisation), 10 DBA
    iterations from it, and the Soft-DTW barycenter of Eq. 7 by 50 Adam steps
    and by L-BFGS (Table I's settings) from it; each scored by the intraclass
    inertia sum_k DTW(B, Y_k) and the
    mean d_score (Eq. 8), the quantities of the paper's barycenter comparison."""
    sb = synth.config_batch(2)
    M = synth.PROTO_LEN[2]
    gb = api.Batch.from_numpy(sb.data, sb.offsets, device=dev)
    B0 = api.euclid_mean(gb, M)
    ws = api.Workspace(dev)

    def quality(B):
        score, cost, _ = api.anomaly_score(B, gb, ws=ws)
        return {"inertia": float(cost.double().sum()), "mean_d_score": float(score.double().mean())}

    res = {"workload": "64 cycles x 1 ch FP32, pre-gap N ~ U(8k,12k), 2% gaps, M=10000",
           "euclidean_mean": quality(B0)}
    barrier()
    t0 = time.perf_counter()
    B = B0.clone()
    for _ in range(dba_iters):
        B, _, _, _ = api.dba_iterate(B, gb, ws=ws)
    barrier()
    res["dba"] = dict(quality(B), iterations=dba_iters, seconds=time.perf_counter() - t0)
    for gamma in gammas:
        t0 = time.perf_counter()
        Bs, hist = api.softdtw_barycenter(gb, M, gamma, steps=steps, lr=lr, init=B0)
        barrier()
        el = time.perf_counter() - t0
        obj = (hist.double().cpu().numpy() * (1.0 / sb.lengths).astype(np.float32)).sum(1)
        res[f"softdtw_barycenter_gamma_{gamma:g}"] = dict(quality(Bs), adam_steps=steps, lr=lr, seconds=el,
                                                          objective_first=float(obj[0]),
                                                          objective_last=float(obj[-1]))
        # the paper's optimiser: L-BFGS with Table I's settings
        t0 = time.perf_counter()
        Bl, f, it, ev, why = api.softdtw_barycenter_lbfgs(gb, M, gamma, init=B0)
        barrier()
        el = time.perf_counter() - t0
        res[f"softdtw_barycenter_lbfgs_gamma_{gamma:g}"] = dict(quality(Bl), iterations=it, evaluations=ev,
                                                                stop=why, objective_last=f, seconds=el)
    # Table I's whole setting: gamma 1, Sakoe-Chiba band 0.6, L-BFGS
    t0 = time.perf_counter()
    Bl, f, it, ev, why = api.softdtw_barycenter_lbfgs(gb, M, 1.0, init=B0, opts=api.options(band=0.6))
    barrier()
    res["softdtw_barycenter_lbfgs_gamma_1_band_0.6"] = dict(quality(Bl), iterations=it, evaluations=ev, stop=why,
                                                            objective_last=f, seconds=time.perf_counter() - t0)
    del ws
    return res


def per_pair_align_ms(api, torch, dev, B, b, gb, barrier):
    """dtw_align launched once per cycle (the plain one-pair-per-launch form)."""
    singles = []
    for k in range(b.T):
        o0, o1 = int(b.offsets[k]), int(b.offsets[k + 1])
        singles.append(api.Batch(gb.data[o0:o1], torch.tensor([0, o1 - o0], device=dev),
                                 np.array([0, o1 - o0], dtype=np.int64)))
    ws = api.Workspace(dev)
    api.dtw_align(B, singles[0], ws=ws)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for one in singles:
        api.dtw_align(B, one, ws=ws)
    e1.record()
    barrier()
    return e0.elapsed_time(e1)


def segment_leg(api, torch, dev, barrier, K: int = 36, cpu_window: bool = True):
    """Segmentation into cycles (Sec. 3.2) in the paper's setting: a
    reference cycle of ~16,300 samples x 9 channels, a stream of K cycles
    (pre-gap U(15k, 18k), ~6e5 samples), windows of 2M, alpha = 0.15 M.  The
    whole loop (one Sub-DTW launch pair per window, the window bounds read
    back each time) is timed from the host, for 16, 8 and 4 rows per lane; one
    2M-column window is also timed on the device, and once by the oracle on
    the host (the CPU baseline of this leg)."""
    import oracle
    X, Y, bounds = synth.segmentation_stream(K, 15000, 18000, 9, 16630, synth.SEED_BASE + 5)
    M, N = len(X), len(Y)
    alpha = int(0.15 * M)
    Xt, Yt = torch.from_numpy(X).to(dev), torch.from_numpy(Y).to(dev)
    res = {"workload": f"reference {M} x 9 ch, stream {N} samples ({K} cycles, pre-gap U(15k,18k), 2% gaps), "
                       f"windows of 2M, alpha = {alpha}", "M": M, "N": N}
    segs = None
    for rows in (16, 8, 4):
        opt = api.options(rows_per_thread=rows)
        ws = api.Workspace(dev)
        api.segment(Xt, Yt[:4 * M], alpha, opt, ws=ws)            # warm-up
        barrier()
        t0 = time.perf_counter()
        segs = api.segment(Xt, Yt, alpha, opt, ws=ws)
        barrier()
        dt = time.perf_counter() - t0
        # cells: M x window length for every window, following the loop's rule
        cells, pos = 0, 0
        for a, b, c in segs:
            we = min(pos + 2 * M, N)
            cells += M * (we - pos)
            if we == N:
                break
            nxt = b - alpha
            pos = nxt if nxt > pos else b + 1
        win = api.Batch.from_numpy(Y[:2 * M], np.array([0, 2 * M], np.int64), device=dev)
        api.subdtw_align(Xt, win, opt, ws=ws)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            api.subdtw_align(Xt, win, opt, ws=ws)
        e1.record()
        barrier()
        w_ms = e0.elapsed_time(e1) / 3
        res[f"rows_{rows}"] = {"windows": len(segs), "seconds": dt, "s_per_window": dt / len(segs),
                               "gcups": cells / dt / 1e9, "window_2M_device_ms": w_ms,
                               "window_2M_gcups": M * 2 * M / (w_ms * 1e-3) / 1e9}
        del ws
    found = 0
    for a, b, c in segs:
        for s0, s1 in bounds:
            ov = min(b, s1) - max(a, s0) + 1
            if ov >= 0.95 * (b - a + 1) and ov >= 0.90 * (s1 - s0 + 1):
                found += 1
                break
    res["cycles_in_stream"] = len(bounds)
    res["pieces_matching_a_cycle"] = found
    res["paper_context"] = "about 3 s per window step for a 16,300-sample reference (Sec. 4.2, other hardware)"
    if cpu_window:
        t0 = time.perf_counter()
        oracle.subdtw(X, Y[:2 * M], "f64")
        dt = time.perf_counter() - t0
        res["cpu_oracle_window_2M"] = {"seconds": dt, "gcups": M * 2 * M / dt / 1e9, "threads": 1,
                                       "sample": "one 2M-column window, FP64"}
    return res


def band_cells(M: int, lengths, band: float) -> int:
    """Cells inside the Sakoe-Chiba band summed over pairs: per row i the
    columns [ceil((i N - B) / M), floor((i N + B) / M)] clipped to [0, N - 1],
    B = floor(band M N) (integer arithmetic, the kernels' definition)."""
    tot = 0
    i = np.arange(M, dtype=np.int64)
    for N in lengths:
        N = int(N)
        B = M * N if band >= 1 else int(np.floor(band * float(M) * float(N)))
        lo = np.maximum(0, -((B - i * N) // M))          # ceil((iN - B) / M)
        hi = np.minimum(N - 1, (i * N + B) // M)
        tot += int(np.maximum(hi - lo + 1, 0).sum())
    return tot


def banded_dba_leg(api, torch, dev, barrier, gb, b, B0, band: float = 0.6, iters: int = 3):
    """One DBA iteration with Table I's Sakoe-Chiba band (0.6) on the benchmark
    batch: time, cells inside the band, and GCUPS over those cells."""
    opt = api.options(band=band)
    ws = api.Workspace(dev)
    B = B0.clone()
    api.dba_iterate(B, gb, opt, ws=ws)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(iters):
        api.dba_iterate(B, gb, opt, ws=ws)
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1) / iters
    cells = band_cells(int(B0.shape[0]), b.lengths, band)
    full = int(B0.shape[0]) * int(b.lengths.sum())
    return {"band": band, "cells_in_band": cells, "fraction_of_matrix": cells / full, "ms_per_dba_iter": ms,
            "gcups_in_band": cells / (ms * 1e-3) / 1e9, "device_status": api.read_status(ws.buf)}


def l2_cost_leg(api, torch, dev, st, barrier, gb, B0, cells: int, ws, iters: int = 2):
    """The l2-norm local cost (cost_kind 1, Sec. 3.2's wording) on the benchmark
    batch: one DBA iteration and one anomaly-score pass, GCUPS over the full
    matrices (the kernels take the IEEE square root of every cell's sum)."""
    opt = api.options(cost_kind=1)
    B = B0.clone()
    api.dba_iterate(B, gb, opt, ws=ws)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(iters):
        api.dba_iterate(B, gb, opt, ws=ws)
    e1.record(st)
    barrier()
    dba_ms = e0.elapsed_time(e1) / iters
    api.anomaly_score(B, gb, opt, ws=ws)
    barrier()
    e0.record(st)
    api.anomaly_score(B, gb, opt, ws=ws)
    e1.record(st)
    barrier()
    sc_ms = e0.elapsed_time(e1)
    return {"cost_kind": 1, "ms_per_dba_iter": dba_ms, "dba_gcups": cells / (dba_ms * 1e-3) / 1e9,
            "anomaly_score_gcups": cells / (sc_ms * 1e-3) / 1e9, "device_status": api.read_status(ws.buf)}


def small_dba_leg(api, torch, dev, barrier, cpu_sample: bool = True):
    """The small DBA workload end to end: 16 cycles of 1.0-1.2k, the medoid
    (pairwise DTW on the GPU) as the start, 10 DBA iterations, then the
    scores; s per iteration from CUDA events; the one-pair-per-launch
    alignment of the same batch; the oracle's iteration on the host."""
    import oracle
    ncores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
    from paper_2404_12134_gb300 import _abi
    b = synth.config_batch(0)
    gb = api.Batch.from_numpy(b.data, b.offsets, device=dev)
    ws = api.Workspace(dev)
    # launch shape for this small batch (untimed; cached): 32 rows per lane
    # give 2 bands per pair, fewer rows more and shorter bands
    idx, _ = api.medoid(api.pairwise_dtw(gb, ws=ws))
    Bw = gb.data[int(b.offsets[int(idx)]):int(b.offsets[int(idx) + 1])].clone()
    dopt, _ = api.autotune(_abi.OP_DBA_ITERATE, Bw, gb, ws)
    sopt, _ = api.autotune(_abi.OP_ANOMALY_SCORE, Bw, gb, ws)
    for _ in range(2):                       # warm-up of the whole workflow
        idx, _ = api.medoid(api.pairwise_dtw(gb, ws=ws))
        Bw = gb.data[int(b.offsets[int(idx)]):int(b.offsets[int(idx) + 1])].clone()
        api.dba_iterate(Bw, gb, dopt, ws=ws)
        api.anomaly_score(Bw, gb, sopt, ws=ws)
    barrier()
    t0 = time.perf_counter()
    idx, _ = api.medoid(api.pairwise_dtw(gb, ws=ws))
    k = int(idx)
    B = gb.data[int(b.offsets[k]):int(b.offsets[k + 1])].clone()
    M0 = B.shape[0]
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        B, _, _, _ = api.dba_iterate(B, gb, dopt, ws=ws)
    e1.record()
    score, cost, _ = api.anomaly_score(B, gb, sopt, ws=ws)
    barrier()
    total = time.perf_counter() - t0
    cells0 = M0 * int(b.lengths.sum())
    it_ms = e0.elapsed_time(e1) / 10
    pp_ms = per_pair_align_ms(api, torch, dev, B, b, gb, barrier)
    res = {"workload": "16 cycles x 1 ch FP32, pre-gap N ~ U(1000,1200), 2% gaps, medoid start, 10 DBA "
                       "iterations + scores", "M": M0, "cells_per_iter": cells0, "s_per_dba_iter": it_ms * 1e-3,
           "gcups": cells0 / (it_ms * 1e-3) / 1e9, "medoid_10_iterations_scores_s": total,
           "per_pair_align_s_per_iter": pp_ms * 1e-3, "device_status": api.read_status(ws.buf),
           "options": {"dba_rows_per_thread": dopt.rows_per_thread, "dba_warps_per_block": dopt.warps_per_block,
                       "score_rows_per_thread": sopt.rows_per_thread,
                       "score_form": "codes + walk" if sopt.score_via_codes else "count inside the DP"}}
    if cpu_sample:
        # the oracle's inputs come from the generator only (its time does not
        # depend on the prototype's values): the first cycle as the prototype
        B_or = b.cycle(0)
        t1 = time.perf_counter()
        oracle.dba_iterate(B_or.astype(np.float64), b.data, b.offsets, "f64")
        cpu_s = time.perf_counter() - t1
        res.update(cpu_oracle_s_per_iter=cpu_s, cpu_oracle_gcups=cells0 / cpu_s / 1e9, cpu_oracle_threads=ncores)
    del ws
    return res


def table_leg(api, torch, dev, barrier):
    """Entries of the results table not covered by the other legs: the small
    DBA workload end to end (medoid init, 10 DBA iterations, scores), the
    one-pair-per-launch form of the two DBA workloads, and the CPU oracle on
    bounded samples of the soft-DTW and uneven-scoring workloads."""
    import oracle
    ncores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
    res = {}
    # workload 0: 16 cycles x 1.0-1.2k, medoid init, 10 DBA iterations + scores
    b = synth.config_batch(0)
    gb = api.Batch.from_numpy(b.data, b.offsets, device=dev)
    ws = api.Workspace(dev)
    barrier()
    t0 = time.perf_counter()
    idx, _ = api.medoid(api.pairwise_dtw(gb, ws=ws))
    k = int(idx)
    B = gb.data[int(b.offsets[k]):int(b.offsets[k + 1])].clone()
    M0 = B.shape[0]
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        B, _, _, _ = api.dba_iterate(B, gb, ws=ws)
    e1.record()
    score, cost, _ = api.anomaly_score(B, gb, ws=ws)
    barrier()
    total = time.perf_counter() - t0
    cells0 = M0 * int(b.lengths.sum())
    it_ms = e0.elapsed_time(e1) / 10
    pp_ms = per_pair_align_ms(api, torch, dev, B, b, gb, barrier)
    t1 = time.perf_counter()
    oracle.dba_iterate(b.cycle(0).astype(np.float64), b.data, b.offsets, "f64")
    cpu_s = time.perf_counter() - t1
    res["small_dba"] = {"M": M0, "cells_per_iter": cells0, "s_per_dba_iter": it_ms * 1e-3,
                        "gcups": cells0 / (it_ms * 1e-3) / 1e9, "workflow_s": total,
                        "per_pair_align_s_per_iter": pp_ms * 1e-3,
                        "cpu_oracle_s_per_iter": cpu_s, "cpu_oracle_gcups": cells0 / cpu_s / 1e9, "cores": ncores}
    del ws
    # workload 1: one-pair-per-launch alignment (the dominant part of a DBA iteration)
    b1, subset = make_workload(200)
    gb1 = api.Batch.from_numpy(b1.data, b1.offsets, device=dev)
    B1 = torch.from_numpy(synth.clean_prototype(b1, M_PROTO)).to(dev)
    pp1 = per_pair_align_ms(api, torch, dev, B1, b1, gb1, barrier)
    cells1 = M_PROTO * int(b1.lengths.sum())
    res["batched_dba_per_pair_align"] = {"ms": pp1, "gcups": cells1 / (pp1 * 1e-3) / 1e9}
    del gb1
    # CPU oracle: soft-DTW fwd + bwd on 4 cycles of workload 2, scoring on 16 of workload 3
    b2 = synth.config_batch(2)
    sub = b2.subset(np.arange(4))
    B2 = synth.clean_prototype(b2, synth.PROTO_LEN[2])
    t1 = time.perf_counter()
    oracle.softdtw_batch(B2, sub.data, sub.offsets, 1.0)
    s2 = time.perf_counter() - t1
    cells2 = synth.PROTO_LEN[2] * int(sub.lengths.sum())
    res["cpu_oracle_softdtw"] = {"sample": "4 of 64 cycles, forward + backward, FP64", "s": s2,
                                 "gcups": cells2 / s2 / 1e9, "threads": min(4, ncores)}
    b3 = synth.config_batch(3)
    sub3 = b3.subset(np.arange(min(ncores, b3.T)))
    B3 = synth.clean_prototype(b3, synth.PROTO_LEN[3])
    t1 = time.perf_counter()
    oracle.score(B3, sub3.data, sub3.offsets, "f64")
    s3 = time.perf_counter() - t1
    cells3 = synth.PROTO_LEN[3] * int(sub3.lengths.sum())
    res["cpu_oracle_scoring"] = {"sample": f"{sub3.T} of 1000 cycles, FP64", "s": s3, "gcups": cells3 / s3 / 1e9,
                                 "threads": ncores}
    return res


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2404_12134_gb300 import api, build
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    if args.leg == "score":
        def sync():
            torch.cuda.synchronize()
        res = scoring_leg(api, torch, dev, sync, T=args.T if args.T != 200 else None)
        if rank == 0:
            print(json.dumps({"leg": "score", "scoring": res}), flush=True)
        return 0
    if args.leg == "long":
        def sync():
            torch.cuda.synchronize()
        res = long_leg(api, torch, dev, sync)
        if rank == 0:
            print(json.dumps({"leg": "long", "long": res}), flush=True)
        return 0
    if args.leg == "table":
        def sync():
            torch.cuda.synchronize()
        res = table_leg(api, torch, dev, sync)
        if rank == 0:
            print(json.dumps({"leg": "table", "table": res}), flush=True)
        return 0
    if args.leg == "bary":
        def sync():
            torch.cuda.synchronize()
        res = bary_leg(api, torch, dev, sync)
        if rank == 0:
            print(json.dumps({"leg": "bary", "barycenters": res}), flush=True)
        return 0
    if args.leg == "segment":
        def sync():
            torch.cuda.synchronize()
        res = segment_leg(api, torch, dev, sync)
        if rank == 0:
            print(json.dumps({"leg": "segment", "segmentation": res}), flush=True)
        return 0
    if args.leg == "small":
        def sync():
            torch.cuda.synchronize()
        res = small_dba_leg(api, torch, dev, sync)
        if rank == 0:
            print(json.dumps({"leg": "small", "small_dba": res}), flush=True)
        return 0
    if args.leg == "softckpt":
        def sync():
            torch.cuda.synchronize()
        res = softckpt_leg(api, torch, dev, sync, T=min(args.T, 32), scale=args.scale, store_pairs=args.store_pairs)
        if rank == 0:
            print(json.dumps({"leg": "softckpt", "softdtw_checkpoint": res}), flush=True)
        return 0
    if args.leg == "soft":
        def sync():
            torch.cuda.synchronize()
        res = softdtw_leg(api, torch, dev, torch.cuda.current_stream(), sync, T=min(args.T, 64), ckpt=args.soft_ckpt,
                          scale=args.scale)
        if rank == 0:
            print(json.dumps({"leg": "soft", "softdtw": res}), flush=True)
        return 0

    b, subset = make_workload(args.T)
    cells = M_PROTO * int(b.lengths.sum())
    gb = api.Batch.from_numpy(b.data, b.offsets, device=dev)

    # initial prototype (untimed): medoid of a seeded 16-cycle subset, resampled to M
    sub = b.subset(subset)
    gsub = api.Batch.from_numpy(sub.data, sub.offsets, device=dev)
    C = api.pairwise_dtw(gsub, ws=api.Workspace(dev))
    idx, _ = api.medoid(C)
    k = int(idx)
    B0 = api.resample(gsub.data[int(sub.offsets[k]):int(sub.offsets[k + 1])], M_PROTO)
    del C, gsub

    ws = api.Workspace(dev)
    from paper_2404_12134_gb300 import _abi
    opts, _ = api.autotune(_abi.OP_DBA_ITERATE, B0, gb, ws)     # untimed, cached
    B = B0.clone()
    Bn = torch.empty_like(B)
    counts = torch.empty(M_PROTO, dtype=torch.int32, device=dev)
    cb = torch.empty((), dtype=torch.float64, device=dev)
    cost = torch.empty(b.T, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def step():
        nonlocal B, Bn
        api.dba_iterate(B, gb, opts, ws=ws, B_out=Bn, counts=counts, cost_before=cb, cost=cost)
        B, Bn = Bn, B

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else None
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    time.sleep(0.5)
    api.profile_read("")                  # drop earlier records
    api.profile_enable(True)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    barrier()
    api.profile_enable(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    wf_ms, wf_n = api.profile_read("wavefront")
    bt_ms, bt_n = api.profile_read("backtrack")
    av_ms, av_n = api.profile_read("dba_average")
    rest_ms, rest_n = api.profile_read("")
    launches = wf_n + bt_n + av_n + rest_n
    ms = max_over_ranks(ms, world, dev)
    status = api.read_status(ws.buf)
    value = world * cells * args.steps / (ms * 1e-3) / 1e9
    dba_cost = float(cb.item())

    out = {
        "metric": "dtw_gcups_dba_iteration", "value": value, "unit": "GCUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": b.T, "d": b.d, "M": M_PROTO, "cells_per_step": cells,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "options": {"rows_per_thread": opts.rows_per_thread, "warps_per_block": opts.warps_per_block},
                   "l2": "no flush: each step writes ~31 GB of predecessor codes (>> 129 MB L2)"},
        "s_per_dba_iter": ms / args.steps * 1e-3,
        "dba_cost_after_warmup_and_steps": dba_cost,
        "device_status": status,
        "gpu_launches": launches,
        "clocks": clk,
    }

    # roofline of the dominant kernel: the wavefront (2-bit code mode).  Work per
    # cell = 2d + 3 FP32 ops (d subtractions, d fused multiply-adds, two mins,
    # one add); peak = SMs x 128 FP32 lanes x max SM clock.
    d = b.d
    wf_avg_s = wf_ms / max(wf_n, 1) * 1e-3
    ops = cells * (2 * d + 3)
    peak = sms * FP32_LANES_PER_SM * 2.070e9 / 1e12
    achieved = ops / wf_avg_s / 1e12
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOP/s (FP32 lane ops)",
                       "frac": achieved / peak,
                       "traffic": WAVEFRONT_DIRS_DRAM_BYTES_PER_CELL * cells if d == 6 else None,
                       "traffic_note": "bytes per launch, ncu dram__bytes_read+write on 36 cycles scaled by cells",
                       "kernel": f"dtw_wavefront_kernel<D=6,R={opts.rows_per_thread},dirs>",
                       "peak_note": f"{sms} SMs x 128 FP32 lanes x 2070 MHz (max SM clock)"}
    out["kernel_ms_per_step"] = {"wavefront": wf_ms / args.steps, "backtrack": bt_ms / args.steps,
                                 "dba_average": av_ms / args.steps, "other": rest_ms / args.steps}
    out["dp_only_gcups"] = cells / wf_avg_s / 1e9

    # end to end through the C ABI with host buffers: pinned host -> device
    # copy of the cycles and prototype, the iteration, device -> host of the
    # new prototype and the cost, every step inside the timed region
    h_data = torch.from_numpy(b.data).pin_memory()
    h_B = B.cpu().pin_memory()
    h_out = torch.empty_like(h_B).pin_memory()
    h_cost = torch.empty((), dtype=torch.float64).pin_memory()
    d_data = torch.empty_like(gb.data)
    gb_e2e = api.Batch(d_data, gb.offsets, gb.offsets_host)
    d_B = torch.empty_like(B)
    n_e2e = max(2, min(args.steps, 10))

    def e2e_step():
        d_data.copy_(h_data, non_blocking=True)
        d_B.copy_(h_B, non_blocking=True)
        api.dba_iterate(d_B, gb_e2e, opts, ws=ws, B_out=Bn, counts=counts, cost_before=cb, cost=cost)
        h_out.copy_(Bn, non_blocking=True)
        h_cost.copy_(cb, non_blocking=True)

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    barrier()
    e2e_s = time.perf_counter() - t0
    out["e2e"] = {"value": world * cells * n_e2e / e2e_s / 1e9, "unit": "GCUPS",
                  "h2d_bytes_per_step": int(h_data.numel() * 4 + h_B.numel() * 4),
                  "d2h_bytes_per_step": int(h_out.numel() * 4 + 8), "steps": n_e2e}
    del d_data, gb_e2e

    if not args.no_extras:
        # anomaly score on the same batch against the current prototype,
        # autotuned: |pi| counted inside the DP, or stored codes + the walk
        sopt, _ = api.autotune(_abi.OP_ANOMALY_SCORE, B, gb, ws)
        api.anomaly_score(B, gb, sopt, ws=ws)
        barrier()
        s0 = torch.cuda.Event(enable_timing=True); s1 = torch.cuda.Event(enable_timing=True)
        s0.record(st)
        api.anomaly_score(B, gb, sopt, ws=ws)
        s1.record(st)
        barrier()
        out["anomaly_score_gcups"] = cells / (s0.elapsed_time(s1) * 1e-3) / 1e9
        out["anomaly_score_options"] = {"rows_per_thread": sopt.rows_per_thread,
                                        "warps_per_block": sopt.warps_per_block,
                                        "form": "codes + walk" if sopt.score_via_codes else "count inside the DP"}
        # the counting form on the same batch, for comparison
        fopt = api.options()
        api.anomaly_score(B, gb, fopt, ws=ws)
        barrier()
        s0.record(st)
        api.anomaly_score(B, gb, fopt, ws=ws)
        s1.record(st)
        barrier()
        out["anomaly_score_count_in_dp_gcups"] = cells / (s0.elapsed_time(s1) * 1e-3) / 1e9
        out["l2_cost"] = l2_cost_leg(api, torch, dev, st, barrier, gb, B0, cells, ws)

    if not args.no_extras:
        out["measured_peaks_probe"] = {k: api.peak_probe(i) / 1e12 for i, k in
                                       enumerate(("fp32_fma_tops", "fp32_minmax_tops", "mufu_ex2_tops",
                                                  "mufu_lg2_tops", "fp32x2_fma_tops", "fp32_min3_tops"))}
        ex2 = out["measured_peaks_probe"]["mufu_ex2_tops"] * 1e12
        lg2 = out["measured_peaks_probe"]["mufu_lg2_tops"] * 1e12
        # the plain one-pair-per-launch form of the benchmark's alignment
        pp1 = per_pair_align_ms(api, torch, dev, B, b, gb, barrier)
        out["batched_dba_per_pair_align"] = {"ms": pp1, "gcups": cells / (pp1 * 1e-3) / 1e9,
                                             "form": "dtw_align once per cycle, in turn"}
        out["scoring"] = scoring_leg(api, torch, dev, barrier)
        out["softdtw"] = softdtw_leg(api, torch, dev, st, barrier, per_pair=True, peaks={"ex2": ex2, "lg2": lg2})
        out["softdtw_band_0.6"] = softdtw_leg(api, torch, dev, st, barrier, band=0.6)
        out["barycenters"] = bary_leg(api, torch, dev, barrier)
        out["segmentation"] = segment_leg(api, torch, dev, barrier)
        out["banded_dba"] = banded_dba_leg(api, torch, dev, barrier, gb, b, B0)
        out["small_dba"] = small_dba_leg(api, torch, dev, barrier, cpu_sample=rank == 0)
        del ws
        torch.cuda.empty_cache()
        out["long"] = long_leg(api, torch, dev, barrier, cpu_sample=rank == 0, ex2=ex2, lg2=lg2)
        sd = out["softdtw"]
        cells_s = sd["cells"]
        t_mufu = cells_s * (2 / ex2 + 1 / lg2) + cells_s * 3 / ex2          # fwd: 2 ex2 + 1 lg2, bwd: 3 ex2
        t_hbm = cells_s * 8 / (hbm_peak_gbs() * 1e9)                        # R: 4 B written + 4 B read
        t = (sd["fwd_ms"] + sd["bwd_ms"]) * 1e-3
        if t_mufu >= t_hbm:
            sd["roofline"] = {"bound": "mufu", "achieved": cells_s * 6 / t / 1e12,
                              "peak": cells_s * 6 / t_mufu / 1e12, "unit": "TOP/s (MUFU ex2+lg2, 5 ex2 + 1 lg2 per cell)",
                              "frac": t_mufu / t, "traffic": None}
        else:
            sd["roofline"] = {"bound": "hbm", "achieved": cells_s * 8 / t / 1e9, "peak": hbm_peak_gbs(),
                              "unit": "GB/s", "frac": t_hbm / t,
                              "traffic": SOFT_FWD_BWD_DRAM_BYTES_PER_CELL * cells_s,
                              "traffic_note": "bytes per forward + backward, ncu dram__bytes_read+write on the "
                                              "64 cycles cut to an eighth, scaled by cells"}
        sd["hbm_lower_bound_ms"] = t_hbm * 1e3
        sd["mufu_lower_bound_ms"] = t_mufu * 1e3

    if rank == 0 and not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", str(ncores))
        n = min(ncores, b.T)
        # the oracle's inputs come from the generator only (its time does not
        # depend on the prototype's values)
        g, dt, c = oracle_dba_sample(b, synth.clean_prototype(b, M_PROTO), n)
        out["cpu_baseline"] = {"value": g, "unit": "GCUPS", "cores": ncores, "kind": "oracle",
                               "sample": f"{n} of {b.T} cycles, one oracle DBA iteration (FP64), "
                                         f"{dt:.1f} s wall on {ncores} threads"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

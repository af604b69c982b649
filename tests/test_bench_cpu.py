"""Host-side pieces of bench.py, on CPU: the in-band cell count against a
direct count, and the reference arm's JSON line (the oracle timed on the
host cores)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_band_cells_counts_the_band():
    sys.path.insert(0, ROOT)
    import bench
    from oracle import brute
    rng = np.random.default_rng(3)
    for _ in range(40):
        M = int(rng.integers(1, 40))
        lens = [int(rng.integers(1, 40)) for _ in range(int(rng.integers(1, 4)))]
        band = float(rng.uniform(0.0, 1.2))
        want = sum(sum(1 for i in range(M) for j in range(n) if brute.in_band(i, j, M, n, band)) for n in lens)
        assert bench.band_cells(M, np.array(lens), band) == want, (M, lens, band)


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == "dtw_gcups_dba_iteration" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]

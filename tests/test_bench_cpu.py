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


def test_store_pairs_that_fit_picks_the_most_that_fit():
    """The bench sizes soft-DTW's store_pairs by free device memory: the most
    pairs whose workspace (the library's own size) fits, less the margin."""
    import ctypes
    import types
    sys.path.insert(0, ROOT)
    import bench
    from paper_2404_12134_gb300 import _abi, api, build
    build.build()
    lib = _abi.load()
    lengths = [9000, 11000, 5000, 10000]
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)

    class FakeBatch:
        T = len(lengths)

        def c(self):
            b = _abi.wts_batch()
            b.data = 16                       # never dereferenced by the sizing call
            b.offsets = 16
            b.offsets_host = offs.ctypes.data
            b.T = self.T
            b.d = 3
            return b

    def size(op, M, batch, opts):
        n = ctypes.c_size_t(0)
        assert lib.wts_workspace_size(op, M, ctypes.byref(batch.c()), ctypes.byref(opts), ctypes.byref(n)) == 0
        return n.value

    fake_api = types.SimpleNamespace(workspace_size=size, options=api.options)
    M = 10000
    sizes = [size(_abi.OP_SOFTDTW, M, FakeBatch(), api.options(dir_mode=1, store_pairs=s)) for s in range(5)]
    assert sizes == sorted(sizes) and sizes[0] < sizes[1]
    for free_bytes, want in ((sizes[0] + 1, 0), (sizes[2] + 16e9, 2), (sizes[2] + 16e9 - 1, 1), (sizes[4] + 20e9, 4)):
        fake_torch = types.SimpleNamespace(cuda=types.SimpleNamespace(
            empty_cache=lambda: None, mem_get_info=lambda dev, f=free_bytes: (int(f), int(f) * 2)))
        got, need = bench.store_pairs_that_fit(fake_api, fake_torch, None, M, FakeBatch())
        assert got == want, (free_bytes, got, want)
        assert need == (sizes[want] if want else 0)

"""Host-side accounting of bench.py: the algorithmic bytes of the FISTA iteration on the C2
recipe (m = 2n, one left rotation so rows pair up, nnz = 8n - 8) and their agreement with the
committed ncu traffic summary."""

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _counted(m, n, nnz):
    """K1 / K2 bytes counted array by array (FP32 values and vectors, int32 indices and
    pointers, float-float iterates): each orientation of the paired storage holds nnz / 2
    indices and nnz values."""
    idx, val = 4 * (nnz // 2), 4 * nnz
    k1 = idx + val + 4 * (m // 2 + 1) + 4 * n + 4 * m * 4      # row pairs; x; A x_{k-2}, b, A x_{k-1}, r
    k2 = idx + val + 4 * (n + 1) + 4 * m + 3 * 8 * n           # columns; r; x_{k-1}, x_{k-2}, x_k
    return k1, k2


def test_c2_bytes_per_iteration():
    n = 2 ** 24
    assert bench.bytes_per_iteration(2 * n, n, 8 * n - 8) == _counted(2 * n, n, 8 * n - 8)
    k1, k2 = bench.bytes_per_iteration(2 * n, n, 8 * n - 8)
    assert round(k1 / 1e9, 3) == 1.476 and round(k2 / 1e9, 3) == 1.409


def test_unpaired_storage_counts_one_index_per_entry():
    m, n, nnz = 1000, 500, 3000
    k1, k2 = bench.bytes_per_iteration(m, n, nnz, paired=False)
    assert k1 == nnz * 8 + 4 * (m + 1) + 4 * n + 16 * m
    assert k2 == nnz * 8 + 4 * (n + 1) + 4 * m + 24 * n


def test_traffic_summary_uses_the_same_accounting():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    n = 2 ** 24
    k1, k2 = bench.bytes_per_iteration(2 * n, n, 8 * n - 8)
    assert d["algorithmic_bytes_per_launch"] == {"k_fista_k1": k1, "k_fista_k2": k2}
    h1, h2 = bench.bytes_per_iteration(2 ** 24, 2 ** 23, 8 * 2 ** 23 - 8)
    assert d["n23"]["k_fista_k1"]["algorithmic"] == h1 and d["n23"]["k_fista_k2"]["algorithmic"] == h2
    for k in ("k_fista_k1", "k_fista_k2"):
        # measured at the bench's size, within 20% of the algorithmic bytes at both sizes
        assert 0.8 <= d["bytes_per_launch"][k] / d["algorithmic_bytes_per_launch"][k] <= 1.2
        assert 0.8 <= d["n23"][k]["dram"] / d["n23"][k]["algorithmic"] <= 1.2


def test_measured_peak_is_read_from_the_peaks_file():
    peak, kind = bench.measured_hbm_peak()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peak > 1000
    else:
        assert kind == "fallback"


def test_matrix_free_accounting_matches_the_summary():
    """K1 = 20n + 16m and K2 = 32n bytes (the factors' O(m + n) vectors only)."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)["matrix_free_n23"]
    n = 2 ** 23
    assert bench.mf_bytes_per_iteration(2 * n, n) == (20 * n + 32 * n, 32 * n)
    assert (d["k1_algorithmic"], d["k2_algorithmic"]) == bench.mf_bytes_per_iteration(2 * n, n)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        e = json.load(f)["matrix_free_n24"]
    assert (e["k1_algorithmic"], e["k2_algorithmic"]) == bench.mf_bytes_per_iteration(2 ** 25, 2 ** 24)


def test_clock_sampler_parses_samples_and_reasons(tmp_path, monkeypatch):
    """The clocks record from a fake nvidia-smi: median SM clock under load, the maximum, and
    the throttle reasons seen Active in any sample."""
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 1965, 2070, 1101.5, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 1980, 2070, 1190.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 1950, 2070, 1188.2, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo 'garbled line'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    for _ in range(100):
        if len(s.lines) >= 4:
            break
        time.sleep(0.05)
    rec = s.stop()
    assert rec["sm_mhz"] == 1965.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_pcg_iteration_bytes_counted_array_by_array():
    """One pdNCG PCG iteration (FP32 values, paired storage), array by array: both orientations
    of the matrix with their pointers; C1 gathers z (n floats) and reads and writes A p (m
    floats each); C2 gathers A p (m floats), reads z, p, h and writes p, Hp (n floats each); C3
    reads d, p, Hp, M^-1 (n floats each) and the float-float residual (n pairs), writes d, z and
    the residual."""
    n = 2 ** 24
    m, nnz = 2 * n, 8 * n - 8
    mats = 2 * (4 * (nnz // 2) + 4 * nnz) + 4 * (m // 2 + 1) + 4 * (n + 1)
    c1 = 4 * n + 4 * m + 4 * m
    c2 = 4 * m + 3 * 4 * n + 2 * 4 * n
    c3 = 4 * 4 * n + 8 * n + 2 * 4 * n + 8 * n
    assert bench.pcg_bytes_per_iteration(m, n, nnz) == mats + c1 + c2 + c3
    assert round(bench.pcg_bytes_per_iteration(m, n, nnz) / 1e9, 2) == 3.22


def test_matrix_free_pcg_iteration_bytes_counted_array_by_array():
    """One PCG iteration of matrix-free pdNCG (FP32 vectors), array by array: the product sweep
    reads z, p_old, the curvature h and sigma and writes p and Hp (n floats each; the halo's
    re-reads, 2 x 16 of every 2048 entries, are not counted); the update reads p, Hp and M^-1,
    reads and writes d (n floats) and the float-float residual (n pairs), and writes z.  No
    m-vector and no matrix."""
    n = 2 ** 24
    sweep = 4 * 4 * n + 2 * 4 * n
    update = 3 * 4 * n + 2 * 4 * n + 2 * 8 * n + 4 * n
    assert bench.mf_pcg_bytes_per_iteration(n) == sweep + update == 64 * n
    assert round(bench.mf_pcg_bytes_per_iteration(n) / 1e9, 2) == 1.07


def test_batch_step_bytes_counted_array_by_array():
    """One step of the batched kernel for one instance (FP32 values, paired storage, float-float
    vectors as {hi, lo} pairs), array by array: both orientations of the matrix with their
    pointers; the row phase gathers the iterate pair (8n), reads and writes A x as pairs (16m),
    reads b (4m) and writes the residual pair (8m); the column phase gathers the residual
    (8m), reads both iterates and writes the new one (24n)."""
    m, n, nnz = 2 ** 19, 2 ** 18, 8 * 2 ** 18 - 8
    mats = 2 * (4 * (nnz // 2) + 4 * nnz) + 4 * (m // 2 + 1) + 4 * (n + 1)
    rows = 8 * n + 16 * m + 4 * m + 8 * m
    cols = 8 * m + 24 * n
    assert bench.batch_bytes_per_step(m, n, nnz) == mats + rows + cols == 12 * nnz + 38 * m + 36 * n + 8

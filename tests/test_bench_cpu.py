"""Host-side arithmetic of the benchmark (CPU): the useful and executed work
per rhs that the roofline divides by, and the traffic figure read from the
committed ncu summaries (used only while the kernel source is unchanged)."""
import os
import shutil

import pytest

import bench


@pytest.mark.parametrize("N", [2, 4, 16, 64, 128, 256])
def test_useful_macs_closed_form(N):
    """4 N sum_m D_m^2 with D_m = N - |m| over the 2N - 1 transfers is
    4 N (N^2 + (N-1) N (2N-1) / 3); over the transfers m <= 0 it is
    4 N sum_{D=1}^{N} D^2 = 4 N N (N+1) (2N+1) / 6."""
    assert bench.contraction_macs(N) == 4 * N * (N * N + (N - 1) * N * (2 * N - 1) // 3)
    assert bench.contraction_macs(N, half=True) == 4 * N * N * (N + 1) * (2 * N + 1) // 6


def test_executed_tensor_work_at_n128():
    """N = 128: 7872 k-steps of 64 complex rows x 128 columns; 3xTF32 issues
    12 MMAs of 128 x 128 x 8 per k-step (24.8 GFLOP), BF16x3 12 of
    128 x 128 x 16 (twice that); the reversal reduction contracts 3968 k-steps."""
    per_kstep_tf32 = 12 * 2 * 128 * 128 * 8
    assert bench.executed_tensor_flops(128) == 7872 * per_kstep_tf32
    assert bench.executed_tensor_flops(128, products=6) == 2 * 7872 * per_kstep_tf32
    assert bench.executed_tensor_flops(128, half=True) == 3968 * per_kstep_tf32


def test_executed_work_bounds_useful_work():
    """Executed tensor flops are at least 3 (3xTF32) or 6 (BF16x3) times the
    useful real flops (8 per complex MAC): the split products of the real
    form, plus padding of ragged transfers to whole tiles."""
    for N in (16, 34, 64, 128):
        useful = 8 * bench.contraction_macs(N)
        assert bench.executed_tensor_flops(N) >= 3 * useful
        assert bench.executed_tensor_flops(N, products=6) >= 6 * useful


@pytest.mark.parametrize("kind", ["tf32", "bf16x3"])
def test_profiled_traffic_follows_the_source_hash(kind, tmp_path, monkeypatch):
    """The committed summary's DRAM bytes are reported while the kernel source
    hashes to the recorded value, and dropped (None) once it differs."""
    import hashlib
    summary = os.path.join(bench.ROOT, "profiles", "contraction_%s_N128.md" % kind)
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    src_rel = os.path.join("paper_1510_07799_gb300", "csrc", "frg_tc.cu")
    (root / os.path.dirname(src_rel)).mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, src_rel), root / src_rel)
    digest = hashlib.sha256(open(root / src_rel, "rb").read()).hexdigest()
    # the committed summary, pointed at this copy of the source
    lines = []
    for line in open(summary):
        if line.startswith("source_sha256:"):
            line = "source_sha256: %s\n" % digest
        lines.append(line)
    (root / "profiles" / os.path.basename(summary)).write_text("".join(lines))
    monkeypatch.setattr(bench, "ROOT", str(root))
    value = bench.profiled_traffic(kind)
    assert value is not None and 5e7 < value < 1e8  # tens of MB per rhs at N = 128
    with open(root / src_rel, "a") as f:
        f.write("\n// changed\n")
    assert bench.profiled_traffic(kind) is None


def test_oracle_baseline_keeps_every_host_core_busy():
    """The oracle's OpenMP loop runs over the vertex rows of one call: the CPU
    baseline and the reference arm hand it two rows per thread (capped at N)."""
    import bench
    assert bench.oracle_rows_per_call(16) == 32
    assert bench.oracle_rows_per_call(1) == 2
    assert bench.oracle_rows_per_call(256, N=128) == 128
    for t in (1, 3, 8, 16, 72):
        assert bench.oracle_rows_per_call(t) >= min(128, 2 * t)

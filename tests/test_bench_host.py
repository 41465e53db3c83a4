"""Host-side logic of the benchmark that needs no GPU: algorithmic bytes,
the variant key and the lookup of committed ncu traffic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_bytes_per_cell():
    # one read and one write of 3 x Q populations and of X at the method's
    # precision: 160 B per species-update (D3Q19 FP32), 84 B (16-bit storage)
    assert bench.bytes_per_cell(3, "fp32") == 3 * 160 == 480
    assert bench.bytes_per_cell(3, "fp16") == 3 * 84 == 252
    assert bench.bytes_per_cell(2, "fp64") == 3 * (2 * 9 * 8 + 16) == 480
    assert bench.bytes_per_cell(2, "fp32") == 3 * 80


def test_variant_key_and_traffic_lookup(tmp_path, monkeypatch):
    info = type("I", (), dict(tile_cells=64, tile_min_blocks=8, threads_per_cell=1, neighbour_bits=32))()
    key = bench.variant_key(info)
    assert key == "64x8/t1/nb32"
    rowmask = type("I", (), dict(tile_cells=64, tile_min_blocks=8, threads_per_cell=1, neighbour_bits=1))()
    assert bench.variant_key(rowmask) == "64x8/t1/nb1"
    sha = bench.kernel_source_sha()
    assert len(sha) == 16 and sha == bench.kernel_source_sha()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text(
        "# comment\n"
        f"kernel_sha={sha} workload=w precision=fp32 variant={key} dram_bytes_per_launch=123\n"
        f"kernel_sha=0000000000000000 workload=w precision=fp16 variant={key} dram_bytes_per_launch=7\n")
    # the lookup reads profiles/ under ROOT and hashes the sources under ROOT
    src = os.path.join(ROOT, "paper_1809_01600_gb300")
    os.symlink(src, tmp_path / "paper_1809_01600_gb300")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("w", "fp32", key) == 123.0
    assert bench.ncu_traffic("w", "fp32", "32x8/t3/nb16") is None      # another variant
    assert bench.ncu_traffic("w", "fp16", key) is None                 # stale kernel hash
    assert bench.ncu_traffic("other", "fp32", key) is None


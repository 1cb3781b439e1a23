"""Host-side arithmetic of bench.py (no GPU)."""
import bench


def test_whole_job_mlups_counts_every_replica():
    # two ranks of 1e6 nodes, 10 steps each, slowest rank 20 ms: 1000 MLUPS
    assert abs(bench.whole_job_mlups(1_000_000, 10, 2, 20.0) - 1000.0) < 1e-9


def test_dram_throughput_helper():
    r = bench.dram_throughput(2.8e9, 0.5, 7000.0)
    assert abs(r["gbs"] - 5600.0) < 1e-9 and abs(r["frac"] - 0.8) < 1e-12
    assert bench.dram_throughput(None, 0.5, 7000.0) is None
    assert bench.dram_throughput(2.8e9, 0.0, 7000.0) is None


def test_algorithmic_bytes_per_node():
    # D3Q19 FP32: phi kernel 2 x 19 x 4 + 2 x 4 = 160 B, composition kernel 152 B
    assert bench.algorithmic_bytes(19, 4, 4) == (160, 152)
    # FP32 arithmetic with 16-bit storage: 84 and 76 B
    assert bench.algorithmic_bytes(19, 4, 2) == (84, 76)

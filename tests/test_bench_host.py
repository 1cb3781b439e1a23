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


def test_compact_legs_and_shared_config():
    import bench
    from paper_2111_05960_gb300 import workloads as WL
    m = WL.recipe(8, 8, 8, D_l=0.1, D_s=0.0, W=3.0)
    cfg = bench.workload_config(m)
    assert cfg["workload"] == "porous_3d_8_d3q19" and cfg["nodes"] == 512
    out = {"value": 16100.0, "roofline": {"kernel": "k_c_step", "frac": 0.71234, "step": {"frac": 0.75},
                                         "kernel_ms": {"k_c_step": 0.5}},
           "batch_2d": {"mlups": 25300.0, "frac": 0.57}, "dev16": {"fp16dev": {"mlups": 14600.0, "step_frac": 0.35}},
           "adjoint": {"adjoint_to_forward": 3.0}}
    legs = bench.compact_legs(out)
    assert legs["step_glups"] == 16.1 and legs["k_c_step_frac"] == 0.7123
    assert legs["batch_2d_glups"] == 25.3 and legs["fp16dev_glups"] == 14.6 and legs["bf16dev_glups"] is None
    assert legs["adjoint_to_forward"] == 3.0 and legs["fp64_glups"] is None

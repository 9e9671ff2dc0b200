"""Host-side logic of the benchmark (CPU): the kernel names it reports for the library's
kernel-choice codes, and the guard that ties a stored DRAM-traffic figure to the kernel source."""
import json
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_simt_tile_table_matches_the_library():
    """bench.SIMT_TILES lists the SIMT launcher's tile candidates in the launcher's order."""
    src = open(os.path.join(ROOT, "paper_2208_07478_gb300", "csrc", "kernels.cu")).read()
    table = src[src.index("static const TileShape kShapes[] = {"):]
    table = table[:table.index("};")]
    tiles = [tuple(int(x) for x in m) for m in re.findall(r"\{(\d+), (\d+), (\d+)\}", table)]
    assert tiles == [tuple(t) for t in bench.SIMT_TILES]


def test_kernel_names_of_choice_codes():
    assert bench.kernel_name(102, "float") == "tc_zgemm_bulk_kernel"
    assert bench.kernel_name(100, "float") == "tc_zgemm_tma_kernel"
    assert bench.kernel_name(200, "double") == "zgemm_smallm_kernel"
    assert bench.kernel_name(3, "double") == "zgemm_kernel<double, 2, 4, 16>"
    assert bench.kernel_name(8013, "double") == "zgemm_kernel<double, 11, 2, 8> split-K 8"
    assert bench.kernel_name(0, "double") == "zgemm_kernel<double>"


def test_stored_traffic_names_its_kernel_and_source():
    info = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    sha = bench.gemm_kernel_sha()
    assert re.fullmatch(r"[0-9a-f]{64}", sha)
    for key in ("kernel", "kernel_step", "precision", "dram_bytes_per_launch", "kernel_source_sha256", "source"):
        assert key in info
    assert os.path.exists(os.path.join(ROOT, info["source"]))
    assert info["dram_bytes_per_launch"] > 0


def test_frequency_walk_covers_the_grid_without_sharing():
    """Each rank walks its own residue class of the frequency grid."""
    nomega, world = 64, 4
    seen = {}
    for rank in range(world):
        for step in range(nomega // world):
            w = bench.omega_index(rank, world, step, nomega)
            assert w not in seen
            seen[w] = rank
    assert sorted(seen) == list(range(nomega))


def test_step_points_of_the_large_meshes_are_distinct():
    """One (k, w) batch per step on the large meshes: every rank and step gets its own pair."""
    nk, nomega, world = 27, 128, 4
    seen = set()
    for rank in range(world):
        for step in range(40):
            p = bench.step_point(rank, world, step, nk, nomega, "one_k")
            assert 0 <= p[0] < nk and 0 <= p[1] < nomega
            assert p not in seen
            seen.add(p)
    assert bench.step_point(0, 1, 5, 8, 64, "all_k") == (-1, 5)


def test_every_workload_has_a_bench_profile():
    from paper_2208_07478_gb300.synth import WORKLOADS
    assert set(bench.PROFILE) == set(WORKLOADS)
    assert bench.WORKLOAD in WORKLOADS


def test_vector_roofline_names_the_binding_resource():
    """The vector steps' bound is whichever of HBM bytes and FP64 flops needs the longer minimum time."""
    hbm = bench.measured_peaks().get("hbm_gbs", 6800.0)
    # 1 GB and 0.01 GFLOP in 1 ms: HBM-bound
    s = {"vector_ms": 1.0, "vector_bytes": 1e9, "vector_flops": 1e7, "vector_gbs": 1e9 / 1e-3 / 1e9,
         "vector_tflops": 1e7 / 1e-3 / 1e12}
    r = bench.vector_roofline(s)
    assert r["bound"] == "hbm"
    assert abs(r["frac_of_bound"] - (1e9 / (hbm * 1e9)) / 1e-3) < 1e-4   # reported to 4 decimals
    # 0.1 GB and 1 GFLOP in 1 ms: FP64-bound on this part
    s = {"vector_ms": 1.0, "vector_bytes": 1e8, "vector_flops": 1e9, "vector_gbs": 100.0, "vector_tflops": 1.0}
    r = bench.vector_roofline(s)
    assert r["bound"] == "alu"
    assert abs(r["frac_of_bound"] - (1e9 / (bench.FP64_PEAK_TFLOPS * 1e12)) / 1e-3) < 1e-4
    assert bench.vector_roofline({"vector_ms": 0.0})["gbs"] is None


def test_every_workload_names_its_refinement():
    for name, cfg in bench.PROFILE.items():
        assert cfg["refine"] in ("fp64", "fp64_tc"), name
        assert cfg["form"] in ("fp64", "tf32x3", "fp32"), name


def test_default_steps_come_from_the_workload(monkeypatch):
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert a.steps is None and a.workload == bench.WORKLOAD
    assert bench.PROFILE[bench.WORKLOAD]["steps"] >= 1

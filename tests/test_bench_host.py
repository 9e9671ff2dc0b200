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

"""The benchmark's roofline inputs come from committed summaries under profiles/: the algorithmic flop counts per
zone-stage and per face (written by oracle/count_stage_flops.py) and the face solve's DRAM bytes per launch
(scaled from an ncu capture).  They parse, are positive, and agree with the per-unit figures they are built
from (the face count of a 256^3 launch without the corner columns is (n + 1)(n^2 + 12 n))."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_stage_flops_and_face_traffic_parse():
    sf = bench.read_stage_flops(256)
    assert sf is not None
    zone = sf["flops_per_zone_stage"]
    face = sf["face_solve_flops_per_face"]
    assert 1000.0 < zone < 1e5 and 100.0 < face < zone
    kv = bench.read_kv("faces_torus_jet_256_traffic.txt")
    n = 256
    faces = (n + 1) * (n * n + 12 * n)
    assert faces == 17632256
    assert abs(kv["dram_bytes_per_launch"] - kv["dram_bytes_per_face"] * faces) <= 1e-3 * kv["dram_bytes_per_launch"]
    assert bench.read_traffic(256) == kv["dram_bytes_per_launch"]
    assert bench.read_traffic(12345) is None

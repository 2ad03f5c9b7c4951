"""Host checks of the benchmark's accounting (no GPU): the algorithmic bytes
per cell that the roofline divides by follow the geometry planes the kernels
actually stage (the plane enum of the library's internal header), and the
replica aggregation divides the right totals."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def geometry_planes():
    src = open(os.path.join(ROOT, "paper_2607_10809_b300", "csrc", "internal.h")).read()
    return {k: int(v) for k, v in re.findall(r"\b(G_[A-Z0-9]+|NRGEO)\s*=\s*(\d+)", src)}


def test_algorithmic_bytes_follow_the_staged_planes():
    g = geometry_planes()
    recon_planes = g["G_IH"] + 1                 # Step-1/2 operators, weights, vertices, moments, 1/h0
    edge_planes = g["G_INR"] + 1 - g["G_NRM"]    # normals, |e|/|K|, inradius
    assert (recon_planes, edge_planes) == (76, 10)
    for s in (4, 8):
        m = 4
        comp = 2 * m * 4 if s == 4 else 0        # FP32: compensation words read and written
        assert bench.alg_bytes("recon", s) == (3 * m + recon_planes + 6 * 3 * m) * s + 3 * 4
        assert bench.alg_bytes("edge", s) == (6 * 3 * m + m + edge_planes + 3 * m) * s + 4 * 4 + comp
    # the per-cell totals quoted for the FP32 step
    assert bench.alg_bytes("recon", 4) == 652 and bench.alg_bytes("edge", 4) == 440
    assert bench.alg_bytes("recon", 4) + bench.alg_bytes("edge", 4) == 1092


def test_replica_value_is_the_whole_job_rate():
    # N ranks each advancing `cells` triangles `steps` times in the slowest rank's time
    v = bench.replicas_value(1_000_000, 10, 5.0, 4)
    assert abs(v - 4 * 1_000_000 * 10 / 5.0e-3) < 1e-6 * v

"""The benchmark's roofline arithmetic on a made-up kernel profile (no GPU):
the dominant kernel is the slowest one, its achieved rate is its method
bytes per launch over its mean event time, the fraction is that over the
measured copy peak, the neighbour + force bytes follow the per-particle,
per-cell, per-pair and per-contact table of the method (192 n + 8 c + 8 p +
64 k in mixed precision, 216 n in FP64), and an ncu traffic figure is
reported only while the sources it was taken on are unchanged."""
import math

import pytest

import bench

N, NCELL, P, K = 100_000, 59_319, 260_000, 102_000
COUNTERS = {"npairs": P, "ncontacts": K, "ncell": [39, 39, 39]}
PEAKS = {"hbm_gbs": 6800.0}


def _profile(slowest):
    # kernel times in ms summed over 10 profiled steps
    prof = {k: 0.1 for k in bench.METHOD_BYTES}
    prof[slowest] = 0.3
    return prof, 10


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_dominant_kernel_and_fraction(precision):
    prof, nprof = _profile("k_pairs")
    step_ms = 0.09
    roof, step, per = bench.roofline(prof, nprof, COUNTERS, N, precision, PEAKS, "measured", step_ms)
    assert roof["kernel"] == "k_pairs"
    mode = 0 if precision == "fp64" else 1
    bn, bc, bp, bk = bench.METHOD_BYTES["k_pairs"][mode]
    mb = bn * N + bc * NCELL + bp * P + bk * K
    assert roof["bytes_per_launch"] == mb
    achieved = mb / (0.03e-3) / 1e9          # 0.3 ms over 10 launches
    assert math.isclose(roof["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(roof["frac"], achieved / 6800.0, rel_tol=1e-12)
    assert math.isclose(roof["share"], 0.3 / (0.1 * (len(prof) - 1) + 0.3), rel_tol=1e-12)
    # the whole step's method bytes over the step time
    total = sum(per[k]["method_bytes"] for k in per)
    assert math.isclose(step["achieved"], total / (step_ms * 1e-3) / 1e9, rel_tol=1e-12)


@pytest.mark.parametrize("precision,bn", [("mixed", 192), ("fp64", 216)])
def test_neighbour_force_bytes_follow_the_method_table(precision, bn):
    prof, nprof = _profile("k_enumerate")
    _, step, _ = bench.roofline(prof, nprof, COUNTERS, N, precision, PEAKS, "measured", 0.5)
    want = bn * N + 8 * NCELL + 8 * P + 64 * K
    assert math.isclose(step["neighbour_force_bytes_per_particle_step"], want / N, rel_tol=1e-12)
    assert math.isclose(step["neighbour_force_frac"], want / 0.5e-3 / 1e9 / 6800.0, rel_tol=1e-12)


def test_traffic_only_for_unchanged_sources():
    for (kernel, precision, n), (traffic, files, digest) in bench.NCU_TRAFFIC.items():
        prof, nprof = _profile(kernel)
        roof, _, _ = bench.roofline(prof, nprof, COUNTERS, n, precision, PEAKS, "measured", 0.1)
        want = traffic if bench.src_hash(files) == digest else None
        assert roof["traffic"] == want, (kernel, n)
    # no record for this size: no traffic figure
    prof, nprof = _profile("k_pairs")
    roof, _, _ = bench.roofline(prof, nprof, COUNTERS, 12345, "mixed", PEAKS, "measured", 0.1)
    assert roof["traffic"] is None

"""Host-side arithmetic of bench.py's derived figures (no GPU)."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


LEVELS = [{"nodes": 257 * 257 * 129}, {"nodes": 129 * 129 * 65}, {"nodes": 65 * 65 * 33}]


def test_relaxation_bandwidths(bench):
    # level 1: 456 B per node (27 complex box entries, 54 imaginary parts, z, r, w) in 1 us per launch
    assert bench.ROOFLINE_BYTES_PER_NODE == 456
    assert bench.class_bandwidth("level1_relax", 1.0, LEVELS) == pytest.approx(456 * 129 * 129 * 65 / 1e3)
    # finest level: 14 packed floats + z, r, w = 80 B per node
    assert bench.FINE_RELAX_BYTES_PER_NODE == 80
    assert bench.class_bandwidth("fine_relax", 2.0, LEVELS) == pytest.approx(80 * 257 * 257 * 129 / 2e3)
    assert bench.class_bandwidth("coarsest", 5.0, LEVELS) is None
    assert bench.class_bandwidth("fine_relax", None, LEVELS) is None


def test_unknown_iterations(bench):
    assert bench.unknown_iterations_per_s(2.0, 1000, [70, 72]) == pytest.approx(2.0 * 1000 * 71)


def test_scale_to_workload(bench):
    # 10 s for 100 nodes x 5 iterations, scaled to 1000 nodes x 50 iterations
    assert bench.scale_to_workload(10.0, 100, 5, 1000, 50) == pytest.approx((100 * 5 / 10.0) / (1000 * 50))

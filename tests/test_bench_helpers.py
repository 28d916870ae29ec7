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


def test_cycle_bytes_two_level_v_cycle(bench):
    # 3D, 1000 fine and 125 coarse nodes, one sweep each side, a 2-step coarsest GMRES (selective
    # second pass not counted at eta 0.1).  Per fine node: pre-smoothing 24 (z = D^{-1} b) + 56 (packed
    # row) + 24 (z, r, w) + 40 (x = alpha z, r -= alpha w, no next z) = 144; post-smoothing 56 + 40
    # (residual with D^{-1}) + 56 + 24 + 48 = 224.  Transfers 8 + 8/8 and 8/8 + 16 per fine node.
    # Coarsest per node: 40 (|b|, V_0, z) + 456 (step 0: 432 stencil + z, w + V_0) + 48 (V_1, z)
    # + 464 (step 1) + 32 (x = D^{-1} V y) = 1040.
    pd = {"cycle": "V", "pre_sweeps": [1, 1], "post_sweeps": [1, 1], "coarse_iterations": 2, "kcycle_iterations": 2,
          "reorth_eta": 0.1}
    levels = [{"nodes": 1000}, {"nodes": 125}]
    assert bench.cycle_bytes(levels, pd) == 144 * 1000 + (8 * 1000 + 8 * 125) + 1040 * 125 + (8 * 125 + 16 * 1000) \
        + 224 * 1000
    # classical Gram-Schmidt twice on the coarsest grid adds 2 C + 2 (j + 1) C per node and step
    pd2 = dict(pd, reorth_eta=2.0)
    assert bench.cycle_bytes(levels, pd2) - bench.cycle_bytes(levels, pd) == (32 + 48) * 125

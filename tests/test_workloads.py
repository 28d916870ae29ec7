"""The seeded synthetic inputs follow their stated recipes: grid spacing,
velocity range, points per wavelength, source placement, the absorbing layer
(0 inside, omega on every absorbing face, none on the Neumann surface) and
determinism under a seed.  They hold none of the method's arithmetic."""
import math

import numpy as np
import pytest

from paper_1712_06091_gb300 import workloads as W


def _face(P, axis, side):
    idx = np.arange(P.N)
    stride = int(np.prod(P.n[:axis]))
    k = (idx // stride) % P.n[axis]
    return k == (0 if side == 0 else P.n[axis] - 1)


@pytest.fixture(scope="module")
def layered():
    return W.layered_3d((65, 65, 33))


def test_layered_grid_velocity_and_frequency(layered):
    P = layered
    assert P.h == pytest.approx((0.1, 0.1, 0.1))                 # 6.4 x 6.4 x 3.2 km on 65 x 65 x 33 nodes
    v = 1.0 / P.kappa
    assert v.min() >= 1.5 * 0.85 - 1e-12 and v.max() <= 5.0 * 1.15 + 1e-12
    # 10 points per wavelength at the lowest velocity: 2 pi v_min / (omega h) = 10
    assert 2 * math.pi * v.min() / (P.omega * max(P.h)) == pytest.approx(10.0, rel=1e-12)
    assert P.src == (32, 32, 2)


def test_layered_absorbing_layer(layered):
    P = layered
    g = P.gamma
    assert g.min() >= 0.0
    for axis, side in W.faces_except_surface(3):
        assert g[_face(P, axis, side)].min() >= P.omega * (1 - 1e-12)   # full strength on each absorbing face
    # one wavelength at the face's mean velocity, in whole cells
    v = 1.0 / P.kappa
    for (axis, side), cells in P.meta["layer_cells"].items():
        wavelength = 2 * math.pi * float(np.mean(v[_face(P, axis, side)])) / P.omega
        assert abs(cells * P.h[axis] - wavelength) <= 0.5 * P.h[axis] + 1e-12


def test_seeded_determinism():
    a = W.layered_3d((33, 33, 17))
    b = W.layered_3d((33, 33, 17))
    c = W.layered_3d((33, 33, 17), seed=5)
    assert np.array_equal(a.kappa, b.kappa) and np.array_equal(a.gamma, b.gamma)
    assert not np.array_equal(a.kappa, c.kappa)


def test_marine_spacing_and_snapped_source():
    P = W.marine_2d((513, 513))
    assert P.h == pytest.approx((8.0 / 512, 4.0 / 512))               # 15.625 m and 7.8125 m
    assert P.src == (256, 6)                                            # 50 m snapped to 46.875 m
    v = 1.0 / P.kappa
    assert v.min() >= 1.5 * 0.8 - 1e-12 and v.max() <= 4.5 * 1.2 + 1e-12


def test_constant_medium_recipe():
    P = W.constant_medium((129, 129))
    assert P.h == pytest.approx((1 / 128, 1 / 128))
    assert P.omega == pytest.approx(2 * math.pi * 12.8)
    assert np.all(P.tau1 == 1.0) and np.all(P.kappa == 1.0)
    assert P.meta["layer_cells"] == {f: 10 for f in W.all_faces(2)}     # one wavelength = 10 cells
    for axis, side in W.all_faces(2):
        assert P.gamma[_face(P, axis, side)].min() == pytest.approx(P.omega)


def test_linear_velocity_traveltime_at_and_near_the_source():
    n, h, src = (41, 21), (0.05, 0.05), (20, 3)
    v0, grad = 1.5, 1.0
    tau1 = W.linear_velocity_traveltime(n, h, src, v0, grad)
    j = src[0] + n[0] * src[1]
    assert tau1[j] == pytest.approx(1.0 / (v0 + grad * src[1] * h[1]))
    # horizontal neighbours at the same depth see the same travel time (symmetry)
    assert tau1[j - 3] == pytest.approx(tau1[j + 3], rel=1e-13)


def test_batch_sources_on_the_surface():
    srcs = W.batch_sources((65, 65, 33), 32)
    assert len(srcs) == 32 and len(set(srcs)) > 1
    assert all(0 <= s[0] < 65 and 0 <= s[1] < 65 and 0 <= s[2] < 2 for s in srcs)

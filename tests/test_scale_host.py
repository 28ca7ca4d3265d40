"""CPU tests of the scaled model's host tables (sam_create_model_scaled).

Against the oracle's scaled projection (oracle.scaled_points, Eq. (2) with
A = s R(theta)): integer offsets of every (scale, angle) table bit-exact,
FP32 directions within FP32 rounding, scaled child shifts bit-exact; one
scale of 1 is the rigid model; the scale grid and argument checks.
"""

import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_2112_05576_gb300 as sam
from paper_2112_05576_gb300 import sam as samb


@pytest.mark.parametrize("levels,step,scales", [(3, 1.0, (0.8, 0.1, 5)), (2, 4.0, (0.5, 0.75, 4)),
                                                (1, 7.5, (1.25, 0.0, 1))])
def test_scaled_tables_match_oracle(levels, step, scales):
    tm, _, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, levels, step, scales=scales)
    om = oracle.create_model(tm, 30, 60, levels, step)
    grid = oracle.scale_grid(*scales)
    assert m.num_scales() == len(grid)
    assert [m.scale(j) for j in range(len(grid))] == grid
    for lvl in range(levels):
        pts = m.points(lvl)
        na = m.num_angles(lvl)
        assert na == om.ntheta(lvl)
        for j, s in enumerate(grid):
            for k in sorted({0, 1, na // 4, na // 3, na // 2, na - 1}):
                ox, oy, px, py = m.rotated_points(lvl, j * na + k)
                rox, roy, rpx, rpy = oracle.scaled_points(pts, k, om.dtheta(lvl), s)
                assert np.array_equal(ox, rox) and np.array_equal(oy, roy), (lvl, j, k)
                assert np.allclose(px, rpx, atol=1e-7) and np.allclose(py, rpy, atol=1e-7)
        if lvl + 1 < levels:
            nap = m.num_angles(lvl + 1)
            for j, s in enumerate(grid):
                for kp in range(0, nap, max(1, nap // 11)):
                    assert m.child_shift(lvl, j * nap + kp) == oracle.child_shift_scaled(om, lvl, kp, s)


def test_unit_scale_is_the_rigid_model():
    tm, _, _ = synth.config1_scene()
    a = sam.Model(tm, 30, 60, 3, 1.0)
    b = sam.Model(tm, 30, 60, 3, 1.0, scales=(1.0, 0.0, 1))
    assert b.num_scales() == a.num_scales() == 1 and b.scale(0) == 1.0
    for lvl in range(3):
        for k in (0, 13, 77):
            k = k % a.num_angles(lvl)
            for u, v in zip(a.rotated_points(lvl, k), b.rotated_points(lvl, k)):
                assert np.array_equal(u, v)


def test_scaled_model_argument_errors():
    tm, _, _ = synth.config1_scene()
    for bad in ((1.0, 0.1, 0), (0.0, 0.1, 3), (-1.0, 0.5, 2), (1.0, 0.0, 3), (1.0, -0.1, 3), (8.0, 1.0, 10),
                (1.0, 0.1, 65)):
        with pytest.raises(sam.SamError) as e:
            sam.Model(tm, 30, 60, 3, 1.0, scales=bad)
        assert e.value.status == samb.SAM_ERR_ARG, bad
    L = sam.lib()
    assert L.sam_model_num_scales(None) == 0 and L.sam_model_scale(None, 0) == 0.0
    m = sam.Model(tm, 30, 60, 3, 1.0, scales=(0.9, 0.1, 3))
    assert m.scale(3) == 0.0 and m.scale(-1) == 0.0
    h = ctypes.c_void_p()
    assert L.sam_create_model_scaled(None, 10, 10, 10, ctypes.byref(samb.ModelParams(30, 60, 1, 1.0, 0)), 1.0, 0.1,
                                     2, ctypes.byref(h)) == samb.SAM_ERR_ARG

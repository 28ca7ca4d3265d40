"""CPU tests of the C ABI: the library loads, exports every declared symbol,
validates arguments, and its host-side model builder (no device work)
matches the oracle: integer Eq. (2) offsets and child shifts bit-exact,
FP32 unit directions within FP32 rounding, edge points identical.
"""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_2112_05576_gb300 as sam
from paper_2112_05576_gb300 import sam as samb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "sam.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sam_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = sam.lib()
    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(samb.SIGNATURES), "binding and header disagree"
    assert L.sam_compiled_arch() == 1030


def test_status_strings_and_defaults():
    assert sam.status_str(0) == "ok"
    assert "argument" in sam.status_str(1)
    p = sam.default_detect_params()
    assert (p.step_x, p.step_y, p.neighbourhood, p.top_k, p.precision) == (1, 1, 3, 64, 0)
    mp = samb.ModelParams()
    sam.lib().sam_default_model_params(ctypes.byref(mp))
    assert (mp.low, mp.high, mp.levels, mp.angle_step_deg, mp.polarity) == (30, 60, 3, 1.0, 0)


def test_create_model_argument_errors():
    tm = np.zeros((32, 32), np.uint8)
    tm[8:24, 8:24] = 200
    with pytest.raises(sam.SamError) as e:
        sam.Model(tm, low=30, high=20)
    assert e.value.status == samb.SAM_ERR_ARG
    with pytest.raises(sam.SamError) as e:
        sam.Model(tm, angle_step_deg=0.7)          # 360/0.7 not an integer
    assert e.value.status == samb.SAM_ERR_ARG
    with pytest.raises(sam.SamError) as e:
        sam.Model(tm, levels=3, angle_step_deg=120.0)  # 3 angles, not divisible by 2^(levels-1)
    assert e.value.status == samb.SAM_ERR_ARG
    flat = np.full((32, 32), 90, np.uint8)
    with pytest.raises(sam.SamError) as e:
        sam.Model(flat)
    assert e.value.status == samb.SAM_ERR_EMPTY_MODEL
    L = sam.lib()
    h = ctypes.c_void_p()
    assert L.sam_create_model(None, 10, 10, 10, ctypes.byref(samb.ModelParams(30, 60, 1, 1.0, 0)),
                              ctypes.byref(h)) == samb.SAM_ERR_ARG


@pytest.mark.parametrize("levels,step", [(3, 1.0), (4, 0.5), (1, 7.5)])
def test_model_tables_match_oracle(levels, step):
    if levels == 4:
        tm, _, _, _ = synth.config2_scene(seed=3300, W=400, H=300)
    else:
        tm, _, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, levels, step)
    om = oracle.create_model(tm, 30, 60, levels, step)
    for lvl in range(levels):
        assert m.template_size(lvl) == om.sizes[lvl]
        tx, ty, gx, gy = m.points(lvl)
        otx, oty, ogx, ogy = om.points[lvl]
        order_a = np.lexsort((tx, ty))
        order_b = np.lexsort((otx, oty))
        for a, b in zip((tx, ty, gx, gy), (otx, oty, ogx, ogy)):
            assert np.array_equal(a[order_a], b[order_b])
        nth = m.num_angles(lvl)
        assert nth == om.ntheta(lvl)
        ks = sorted(set([0, 1, nth // 4, nth // 3, nth // 2, nth - 1] + list(range(0, nth, max(1, nth // 23)))))
        for k in ks:
            ox, oy, px, py = m.rotated_points(lvl, k)
            rox, roy, rpx, rpy = oracle.rotate_points((tx, ty, gx, gy), k, om.dtheta(lvl))
            assert np.array_equal(ox, rox) and np.array_equal(oy, roy), (lvl, k)
            assert np.allclose(px, rpx, atol=1e-7) and np.allclose(py, rpy, atol=1e-7)
        if lvl + 1 < levels:
            for kp in range(0, m.num_angles(lvl + 1), max(1, m.num_angles(lvl + 1) // 37)):
                assert m.child_shift(lvl, kp) == oracle.child_shift(om, lvl, kp)

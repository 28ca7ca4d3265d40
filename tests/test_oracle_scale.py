"""Pins of the oracle's scaled-pose search (Eq. (2) with A = s R(theta)).

What fixes it, independently of the oracle's own code:
  * one scale of 1 is exactly the rigid search: the same maps (up to FP64
    rounding of the directions), candidates, refinement and detections;
  * scaling a projection scales its offsets: at 0 and 90 degrees the offsets
    for s = 2 are 2 t and 2 R t exactly, and the directions do not change;
  * the 4-D candidate rule equals a plain numpy brute force over every pose
    and its 80 neighbours on tied maps (so a dropped neighbour, a circular
    scale axis or a wrong tie order fails it);
  * a template enlarged 2x by pixel replication is detected at scale 2 with
    score 1, at 0 and at 90 degrees, by a one-level search and by the
    two-level coarse-to-fine descent (which must carry the scale down).
"""

import itertools

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def cfg1():
    tm, sc, truth = synth.config1_scene()
    om = oracle.create_model(tm, 30, 60, 3, 1.0)
    return tm, sc, om


def test_unit_scale_is_the_rigid_search(cfg1):
    tm, sc, om = cfg1
    top = 2
    field = oracle.search_fields(sc, 3, 30)[top]
    rigid = oracle.score_map(field, om.points[top], om.ntheta(top), om.dtheta(top))
    scaled = oracle.score_map_scaled(field, om.points[top], [1.0], om.ntheta(top), om.dtheta(top))
    assert scaled.shape == (1,) + rigid.shape
    assert np.abs(scaled[0] - rigid).max() < 1e-12
    for k in (0, 7, 45, 89):
        for lvl in (0, 1):
            assert oracle.child_shift_scaled(om, lvl, k, 1.0) == oracle.child_shift(om, lvl, k)
    p = oracle.DetectParams(min_score=0.7)
    ref = oracle.detect(om, sc, p)
    got = oracle.detect_scaled(om, sc, p, [1.0])
    assert len(ref) == len(got) > 0
    for r, g in zip(ref, got):
        assert (r[0], r[1], r[4]) == (g[0], g[1], g[4]) and g[5] == 0
        assert abs(r[3] - g[3]) < 1e-12


def test_scaled_points_scale_the_offsets(cfg1):
    _, _, om = cfg1
    pts = om.points[0]
    tx, ty = pts[0], pts[1]
    for s in (2.0, 3.0):
        ox, oy, px, py = oracle.scaled_points(pts, 0, 1.0, s)
        assert np.array_equal(ox, s * tx) and np.array_equal(oy, s * ty)
        rot = oracle.rotate_points(pts, 0, 1.0)
        assert np.abs(px - rot[2]).max() < 1e-15 and np.abs(py - rot[3]).max() < 1e-15
        # a quarter turn (x right, y down): R t = (-ty, tx)
        ox, oy, px, py = oracle.scaled_points(pts, 90, 1.0, s)
        assert np.array_equal(ox, -s * ty) and np.array_equal(oy, s * tx)
        rot = oracle.rotate_points(pts, 90, 1.0)
        assert np.abs(px - rot[2]).max() < 1e-15 and np.abs(py - rot[3]).max() < 1e-15


def _brute_candidates(smap, min_score, K):
    ns, nth, gh, gw = smap.shape
    found = []
    for j, k, y, x in itertools.product(range(ns), range(nth), range(gh), range(gw)):
        s = smap[j, k, y, x]
        if not s >= min_score:
            continue
        key = ((j * nth + k) * gh + y) * gw + x
        ok = True
        for dj, dk, dy, dx in itertools.product((-1, 0, 1), repeat=4):
            if (dj, dk, dy, dx) == (0, 0, 0, 0):
                continue
            j2, y2, x2 = j + dj, y + dy, x + dx
            if dk != 0 and nth == 1:
                continue
            k2 = (k + dk) % nth
            if not (0 <= j2 < ns and 0 <= y2 < gh and 0 <= x2 < gw):
                continue
            key2 = ((j2 * nth + k2) * gh + y2) * gw + x2
            if key2 == key:
                continue
            s2 = smap[j2, k2, y2, x2]
            if not (s > s2 or (s == s2 and key < key2)):
                ok = False
                break
        if ok:
            found.append((-s, key, j, k, y, x))
    found.sort()
    return found[:K]


@pytest.mark.parametrize("shape", [(1, 4, 5, 6), (3, 1, 4, 4), (2, 3, 5, 4), (4, 5, 3, 3), (3, 2, 6, 5)])
def test_candidates_scaled_equal_brute_force(shape):
    rng = np.random.default_rng(int(np.prod(shape)))
    smap = rng.integers(0, 9, shape) / 8.0
    K = 50
    cj, ck, cy, cx, cs = oracle.candidates_scaled(smap, 0.25, K)
    ref = _brute_candidates(smap, 0.25, K)
    assert len(cj) == len(ref)
    assert [(int(a), int(b), int(c), int(d)) for a, b, c, d in zip(cj, ck, cy, cx)] == [r[2:] for r in ref]
    assert np.array_equal(cs, np.array([-r[0] for r in ref]))
    if shape[0] == 1:   # one scale: the 3-D candidates
        rk, ry, rx, rs = oracle.candidates(smap[0], 0.25, K)
        assert np.array_equal(ck, rk) and np.array_equal(cy, ry) and np.array_equal(cx, rx)


def _enlarged_scene():
    tm = np.full((24, 24), 60, np.uint8)
    tm[6:18, 6:18] = 200
    tm[9:12, 9:15] = 60                          # a slot, so the part is not symmetric
    scene = np.full((80, 80), 60, np.uint8)
    scene[16:64, 16:64] = np.kron(tm, np.ones((2, 2), np.uint8))
    return tm, scene


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("quarter", [0, 1])
def test_enlarged_template_detected_at_scale_two(levels, quarter):
    tm, scene = _enlarged_scene()
    if quarter:
        scene = np.ascontiguousarray(np.rot90(scene, -1))   # turned 90 degrees with y down
    # the top level searches quarter turns (45 degree steps at level 0 with
    # two levels), so the turned instance is on the top-level angle grid
    step = 90.0 if levels == 1 else 45.0
    om = oracle.create_model(tm, 30, 60, levels, step)
    scales = [1.0, 1.5, 2.0, 2.5] if levels == 1 else [1.0, 1.5, 2.0]
    dets = oracle.detect_scaled(om, scene, oracle.DetectParams(min_score=0.5), scales)
    x, y, th, s, k, j = dets[0]
    assert j == 2 and k == quarter * int(90 / step) and abs(s - 1.0) < 1e-12
    # the template's reference pixel covers scene pixels 40..41 (38..39 on
    # the turned scene's x axis)
    assert y in (40, 41) and x in ((40, 41) if not quarter else (38, 39))
    assert all(d[3] <= s for d in dets)


def test_child_shift_of_quarter_turns_in_closed_form():
    # The level-l child of a level-(l+1) pose u' is 2 u' + (1/2, 1/2) - A d,
    # d = 2 c_{l+1} + 1/2 - c_l (c = reference point), rounded half up.  For
    # quarter turns A = s R is exact: R(0) d = d, R(90) d = (-d_y, d_x),
    # R(180) d = -d, R(270) d = (d_y, -d_x), so the shift is known in exact
    # rational arithmetic (here d is +-1/2 per axis).
    from fractions import Fraction as F
    import math
    for side in (24, 26, 27):               # d = +1/2, -1/2, +1/2 per axis
        tm = np.full((side, side), 60, np.uint8)
        tm[5:side - 5, 5:side - 5] = 200
        om = oracle.create_model(tm, 30, 60, 2, 90.0)
        (w0, h0), (w1, h1) = om.sizes
        d = (F(2 * (w1 // 2)) + F(1, 2) - F(w0 // 2), F(2 * (h1 // 2)) + F(1, 2) - F(h0 // 2))
        for k_parent, (rx, ry) in ((0, (d[0], d[1])), (1, (-d[0], -d[1]))):   # level-1 angles 0 and 180
            # scales with s d an integer (s = 2, 4) put the exact child on a
            # rounding tie, which the FP64 evaluation of sin(180 deg) decides
            for s in (F(1), F(5, 4), F(5, 2), F(3), F(7, 2)):
                want = (math.floor(F(1, 2) - s * rx + F(1, 2)), math.floor(F(1, 2) - s * ry + F(1, 2)))
                assert oracle.child_shift_scaled(om, 0, k_parent, float(s)) == want, (side, k_parent, s)

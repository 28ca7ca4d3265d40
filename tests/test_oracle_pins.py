"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: values
computed by hand (tests/golden), closed forms, library routines (scipy),
invariances the paper claims for Eq. (1), and brute force on tiny inputs.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _golden(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# gradients (Sec. II edge extraction)
# ---------------------------------------------------------------------------

def test_sobel_golden(golden_dir):
    g = _golden(golden_dir, "sobel_4x4.json")
    gx, gy = oracle.sobel(np.array(g["image"], np.uint8))
    assert gx.tolist() == g["gx"]
    assert gy.tolist() == g["gy"]


def test_sobel_ramp_closed_form():
    # I = a x + b y + c  =>  interior gx = 8 a, gy = 8 b, border 0
    for a, b, c in [(3, 0, 10), (0, 5, 7), (2, -3, 120), (-4, 1, 200)]:
        ys, xs = np.mgrid[0:12, 0:15]
        img = (a * xs + b * ys + c).astype(np.int64)
        assert img.min() >= 0 and img.max() <= 255
        gx, gy = oracle.sobel(img.astype(np.uint8))
        assert np.all(gx[1:-1, 1:-1] == 8 * a) and np.all(gy[1:-1, 1:-1] == 8 * b)
        for arr in (gx, gy):
            assert np.all(arr[0] == 0) and np.all(arr[-1] == 0) and np.all(arr[:, 0] == 0) and np.all(arr[:, -1] == 0)


def test_sobel_matches_scipy_correlate():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, (37, 53)).astype(np.uint8)
    gx, gy = oracle.sobel(img)
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    ref_x = ndi.correlate(img.astype(np.int64), kx, mode="constant")
    ref_y = ndi.correlate(img.astype(np.int64), kx.T, mode="constant")
    assert np.array_equal(gx[1:-1, 1:-1], ref_x[1:-1, 1:-1])
    assert np.array_equal(gy[1:-1, 1:-1], ref_y[1:-1, 1:-1])


def test_sobel_quarter_turn_equivariance():
    # Turning the image by 90 degrees permutes the interior gradients exactly.
    rng = np.random.default_rng(8)
    img = rng.integers(0, 256, (20, 20)).astype(np.uint8)
    gx, gy = oracle.sobel(img)
    r = np.rot90(img)  # r[i, j] = img[j, W-1-i]: image turned counter-clockwise on screen
    rgx, rgy = oracle.sobel(np.ascontiguousarray(r))
    # r at (x=j, y=i) is img at (x'=W-1-i, y'=j): d/dx of r is d/dy' of img,
    # d/dy of r is -d/dx' of img
    assert np.array_equal(rgx[1:-1, 1:-1], np.rot90(gy)[1:-1, 1:-1])
    assert np.array_equal(rgy[1:-1, 1:-1], -np.rot90(gx)[1:-1, 1:-1])


def test_threshold_units_and_boundary():
    # |g|/4 >= T  <=>  gx^2 + gy^2 >= 16 T^2 ; a step of height h has magnitude h
    T = 30
    gx = np.array([4 * T, 4 * T - 1, 72, 96, 0, -120, 1020], np.int32)
    gy = np.array([0, 0, 96, 72, -120, 1, 1020], np.int32)
    m = oracle.search_mask(gx, gy, T)
    assert m.tolist() == [1, 0, 1, 1, 1, 1, 1]
    rng = np.random.default_rng(3)
    gx = rng.integers(-1020, 1021, 5000).astype(np.int32)
    gy = rng.integers(-1020, 1021, 5000).astype(np.int32)
    mag = np.hypot(gx.astype(float), gy.astype(float)) / 4.0
    m = oracle.search_mask(gx, gy, T)
    clear = np.abs(mag - T) > 1e-6
    assert np.array_equal(m[clear].astype(bool), (mag >= T)[clear])
    # vertical step edge of height h: Sobel magnitude/4 equals h in the interior
    img = np.zeros((8, 8), np.uint8)
    img[:, 4:] = 50
    gx, gy = oracle.sobel(img)
    assert gx[3, 4] // 4 == 50 and gx[3, 3] // 4 == 50


def test_hysteresis_matches_connected_components():
    rng = np.random.default_rng(11)
    for _ in range(5):
        img = ndi.gaussian_filter(rng.normal(128, 60, (48, 64)), 1.5).clip(0, 255).astype(np.uint8)
        gx, gy = oracle.sobel(img)
        low, high = 6, 14
        m = oracle.hysteresis(gx, gy, low, high)
        mag2 = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2
        weak = mag2 >= 16 * low * low
        strong = mag2 >= 16 * high * high
        lab, _ = ndi.label(weak, structure=np.ones((3, 3)))
        keep = np.unique(lab[strong])
        ref = np.isin(lab, keep[keep > 0])
        assert np.array_equal(m.astype(bool), ref)


# ---------------------------------------------------------------------------
# pyramid
# ---------------------------------------------------------------------------

def test_pyramid_golden(golden_dir):
    for case in _golden(golden_dir, "pyramid.json")["cases"]:
        d = oracle.pyramid_down(np.array(case["image"], np.uint8))
        assert d.tolist() == case["down"] or (d.size == 0 and case["down"] == [])


def test_pyramid_rounded_mean_and_constant():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (33, 47)).astype(np.uint8)
    d = oracle.pyramid_down(img)
    blocks = img[:32, :46].astype(np.float64).reshape(16, 2, 23, 2).mean(axis=(1, 3))
    assert np.array_equal(d, np.floor(blocks + 0.5).astype(np.uint8))
    c = np.full((10, 14), 77, np.uint8)
    assert np.all(oracle.pyramid_down(c) == 77)


# ---------------------------------------------------------------------------
# unit field, model points, rotation (Eq. (1) normalisation, Eq. (2))
# ---------------------------------------------------------------------------

def test_unit_field_and_model_points():
    tm, _, _ = synth.config1_scene()
    gx, gy = oracle.sobel(tm)
    mask = oracle.hysteresis(gx, gy, 30, 60)
    f = oracle.unit_field(gx, gy, mask)
    nrm = np.hypot(f[..., 0], f[..., 1])
    assert np.allclose(nrm[mask == 1], 1.0, atol=1e-15) and np.all(nrm[mask == 0] == 0)
    ang = np.arctan2(f[..., 1], f[..., 0])
    ref = np.arctan2(gy, gx)
    assert np.allclose(np.cos(ang - ref)[mask == 1], 1.0, atol=1e-12)
    tx, ty, pgx, pgy = oracle.model_points(tm, 30, 60)
    assert len(tx) == int(mask.sum())
    rows, cols = np.nonzero(mask)
    assert np.array_equal(tx, cols - 24) and np.array_equal(ty, rows - 24)
    assert np.array_equal(pgx, gx[rows, cols]) and np.array_equal(pgy, gy[rows, cols])


def test_rotation_quarter_turns_exact():
    rng = np.random.default_rng(1)
    tx = rng.integers(-30, 31, 50).astype(np.int32)
    ty = rng.integers(-30, 31, 50).astype(np.int32)
    gx = rng.integers(-500, 501, 50).astype(np.int32)
    gy = rng.integers(-500, 501, 50).astype(np.int32)
    gx[gx == 0] = 1
    expect = {0: (tx, ty), 1: (-ty, tx), 2: (-tx, -ty), 3: (ty, -tx)}   # x right, y down, R(theta) of Eq. (2)
    for k, (ex, ey) in expect.items():
        ox, oy, px, py = oracle.rotate_points((tx, ty, gx, gy), k, 90.0)
        assert np.array_equal(ox, ex) and np.array_equal(oy, ey)
        m = np.hypot(gx, gy)
        gex, gey = {0: (gx, gy), 1: (-gy, gx), 2: (-gx, -gy), 3: (gy, -gx)}[k]
        assert np.allclose(px, gex / m, atol=1e-15) and np.allclose(py, gey / m, atol=1e-15)


def test_rotation_general_angle_bounds():
    rng = np.random.default_rng(2)
    tx = rng.integers(-100, 101, 300).astype(np.int32)
    ty = rng.integers(-100, 101, 300).astype(np.int32)
    gx = rng.integers(1, 500, 300).astype(np.int32)
    gy = rng.integers(-500, 500, 300).astype(np.int32)
    for k in [1, 7, 33, 100, 359]:
        th = math.radians(k * 1.0)
        ox, oy, px, py = oracle.rotate_points((tx, ty, gx, gy), k, 1.0)
        rx = math.cos(th) * tx - math.sin(th) * ty
        ry = math.sin(th) * tx + math.cos(th) * ty
        assert np.all(np.abs(ox - rx) <= 0.5 + 1e-9) and np.all(np.abs(oy - ry) <= 0.5 + 1e-9)
        assert np.allclose(np.hypot(px, py), 1.0, atol=1e-14)
        # p_hat is the model gradient turned by theta: its angle grows by theta
        d = np.arctan2(py, px) - np.arctan2(gy, gx)
        assert np.allclose(np.cos(d), math.cos(th), atol=1e-12) and np.allclose(np.sin(d), math.sin(th), atol=1e-12)


# ---------------------------------------------------------------------------
# Eq. (1) with neighbouring search
# ---------------------------------------------------------------------------

def _golden_field(g):
    f = np.zeros((g["h"], g["w"], 2))
    for x, y, wx, wy in g["edges"]:
        f[y, x] = (wx, wy)
    return f


def test_score_golden(golden_dir):
    g = _golden(golden_dir, "score_5x5.json")
    f = _golden_field(g["field"])
    m = g["model"]
    pts = tuple(np.array(m[k], np.int32) for k in ("tx", "ty", "gx", "gy"))
    for c in g["cases"]:
        rot = oracle.rotate_points(pts, c["k"], c["dtheta"])
        assert [[int(a), int(b)] for a, b in zip(rot[0], rot[1])] == c["offsets"]
        M = oracle.score_pose(f, rot, c["u"][0], c["u"][1], c["nbhd"], c["polarity"])
        assert M == pytest.approx(c["M"], abs=1e-12), c


def test_single_point_neighbourhood_window():
    # One edge pixel, one model point: the vote is nonzero exactly on the
    # 3x3 pose window (size 3) or at the one pose (size 1).
    f = np.zeros((9, 9, 2))
    f[4, 4] = (0.6, -0.8)
    pts = (np.array([0], np.int32), np.array([0], np.int32), np.array([3], np.int32), np.array([-4], np.int32))
    smap3 = oracle.score_map(f, pts, 1, 360.0, nbhd=3)[0]
    smap1 = oracle.score_map(f, pts, 1, 360.0, nbhd=1)[0]
    exp3 = np.zeros((9, 9))
    exp3[3:6, 3:6] = 1.0
    exp1 = np.zeros((9, 9))
    exp1[4, 4] = 1.0
    assert np.allclose(smap3, exp3, atol=1e-15) and np.allclose(smap1, exp1, atol=1e-15)


def test_neighbourhood_monotone_and_bounded():
    tm, sc, _ = synth.tiny_case(21, size=28, tsize=9)
    model = oracle.create_model(tm, 10, 20, 1, 30.0)
    f = oracle.search_fields(sc, 1, 10)[0]
    m3 = oracle.score_map(f, model.points[0], 12, 30.0, nbhd=3)
    m1 = oracle.score_map(f, model.points[0], 12, 30.0, nbhd=1)
    assert np.all(m3 >= m1 - 1e-15)
    assert np.all(m3 <= 1 + 1e-12) and np.all(m1 >= -1 - 1e-12)
    p3 = oracle.score_map(f, model.points[0], 12, 30.0, nbhd=3, polarity=1)
    assert np.all(p3 >= m3 - 1e-15) and np.all(p3 >= 0)


def _brute_map(field, pts, ntheta, dtheta, nbhd, polarity):
    """Independent numpy brute force: for each angle and neighbour offset shift
    the whole zero-padded field and accumulate over points."""
    tx, ty, gx, gy = (np.asarray(a, np.float64) for a in pts)
    H, W = field.shape[:2]
    r = nbhd // 2
    pad = 64
    F = np.zeros((H + 2 * pad, W + 2 * pad, 2))
    F[pad:pad + H, pad:pad + W] = field
    out = np.zeros((ntheta, H, W))
    mag = np.hypot(gx, gy)
    for k in range(ntheta):
        th = ((k * dtheta) * math.pi) / 180.0
        c, s = math.cos(th), math.sin(th)
        ox = np.floor(c * tx - s * ty + 0.5).astype(int)
        oy = np.floor(s * tx + c * ty + 0.5).astype(int)
        px = (c * gx - s * gy) / mag
        py = (s * gx + c * gy) / mag
        acc = np.zeros((H, W))
        for i in range(len(tx)):
            best = np.full((H, W), -np.inf)
            for b in range(-r, r + 1):
                for a in range(-r, r + 1):
                    y0, x0 = pad + oy[i] + b, pad + ox[i] + a
                    win = F[y0:y0 + H, x0:x0 + W]
                    v = px[i] * win[..., 0] + py[i] * win[..., 1]
                    if polarity:
                        v = np.abs(v)
                    best = np.maximum(best, v)
            acc += best
        out[k] = acc / len(tx)
    return out


@pytest.mark.parametrize("seed,nbhd,polarity", [(31, 3, 0), (32, 1, 0), (33, 3, 1)])
def test_score_map_brute_force_32(seed, nbhd, polarity):
    tm, sc, _ = synth.tiny_case(seed, size=32, tsize=9)
    model = oracle.create_model(tm, 10, 20, 1, 45.0)
    f = oracle.search_fields(sc, 1, 10)[0]
    got = oracle.score_map(f, model.points[0], 8, 45.0, nbhd=nbhd, polarity=polarity)
    ref = _brute_map(f, model.points[0], 8, 45.0, nbhd, polarity)
    assert np.allclose(got, ref, atol=1e-12)


def test_score_map_step_grid():
    tm, sc, _ = synth.tiny_case(41, size=30, tsize=9)
    model = oracle.create_model(tm, 10, 20, 1, 90.0)
    f = oracle.search_fields(sc, 1, 10)[0]
    full = oracle.score_map(f, model.points[0], 4, 90.0)
    stepped = oracle.score_map(f, model.points[0], 4, 90.0, step_x=3, step_y=2)
    assert stepped.shape == (4, 15, 10)
    assert np.array_equal(stepped, full[:, ::2, ::3])


def _paste_setup(theta, levels=3, side=48, seed=12):
    rng = np.random.default_rng(seed)
    spec = synth.random_part(rng, side, kind="tiny", margin=4.0)
    tmpl = synth.render_template(spec)
    return spec, tmpl


# Hand-derived coarse-to-fine shifts for even template sizes (d = 1/2 per
# axis): shift = (1/2, 1/2) - R(theta) (1/2, 1/2) for theta = 0, 90, 180, 270.
QUARTER_SHIFT = {0: (0, 0), 90: (1, 0), 180: (1, 1), 270: (0, 1)}


@pytest.mark.parametrize("theta", [0, 90, 180, 270])
def test_paste_scores_one_at_every_level(theta):
    """A noise-free template pasted at a pose scores exactly 1 there (every
    cosine is 1), at every pyramid level, and is the best pose of the map."""
    levels = 3
    spec, tmpl = _paste_setup(theta)
    model = oracle.create_model(tmpl, 30, 60, levels, 90.0 / 4)   # 16 angles at level 0
    # choose the top-level pose, derive the lower ones with the hand shifts
    u = [None] * levels
    u[levels - 1] = (19, 17)
    sx, sy = QUARTER_SHIFT[theta]
    for lvl in range(levels - 2, -1, -1):
        u[lvl] = (2 * u[lvl + 1][0] + sx, 2 * u[lvl + 1][1] + sy)
        kp = theta // int(model.dtheta(lvl + 1))
        assert oracle.child_shift(model, lvl, kp) == (sx, sy)
    W = H = 8 * 24
    img = synth.paste_scene(spec, (W, H), [(u[0][0], u[0][1], float(theta))])
    fields = oracle.search_fields(img, levels, 30)
    for lvl in range(levels):
        k = int(theta / model.dtheta(lvl))
        rot = oracle.rotate_points(model.points[lvl], k, model.dtheta(lvl))
        for nb in (1, 3):
            M = oracle.score_pose(fields[lvl], rot, u[lvl][0], u[lvl][1], nb, 0)
            assert M == pytest.approx(1.0, abs=1e-12), (lvl, nb)
    top = levels - 1
    smap = oracle.score_map(fields[top], model.points[top], model.ntheta(top), model.dtheta(top), nbhd=1)
    k = int(theta / model.dtheta(top))
    assert smap[k, u[top][1], u[top][0]] == pytest.approx(1.0, abs=1e-12)
    assert smap.max() <= 1.0 + 1e-12
    # With size-3 neighbouring search every pose within 1 px of the paste also
    # scores 1 (ties go to the smaller key), so the exact pose is checked with
    # size 1, where it is the unique maximum.
    det = oracle.detect(model, img, oracle.DetectParams(min_score=0.8, nbhd=1))
    assert (det[0][0], det[0][1]) == u[0] and det[0][2] == float(theta)
    assert det[0][3] == pytest.approx(1.0, abs=1e-12)
    det3 = oracle.detect(model, img, oracle.DetectParams(min_score=0.8, nbhd=3))
    assert abs(det3[0][0] - u[0][0]) <= 1 and abs(det3[0][1] - u[0][1]) <= 1
    assert det3[0][3] == pytest.approx(1.0, abs=1e-12)


def test_contrast_inversion():
    tm, sc, _ = synth.tiny_case(51, size=32, tsize=9)
    model = oracle.create_model(tm, 10, 20, 1, 45.0)
    f = oracle.search_fields(sc, 1, 10)[0]
    fi = oracle.search_fields(255 - sc, 1, 10)[0]
    assert np.array_equal(fi, -f)
    for nb in (1, 3):
        a = oracle.score_map(f, model.points[0], 8, 45.0, nbhd=nb, polarity=1)
        b = oracle.score_map(fi, model.points[0], 8, 45.0, nbhd=nb, polarity=1)
        assert np.array_equal(a, b)
    a = oracle.score_map(f, model.points[0], 8, 45.0, nbhd=1, polarity=0)
    b = oracle.score_map(fi, model.points[0], 8, 45.0, nbhd=1, polarity=0)
    assert np.array_equal(b, -a)


def test_gain_and_offset_invariance():
    rng = np.random.default_rng(9)
    spec = synth.random_part(rng, 24, kind="tiny", margin=3.0)
    spec.part_level, spec.background = 120.0, 40.0
    tmpl = synth.render_template(spec)
    img = synth.paste_scene(spec, (64, 64), [(30, 33, 0.0)], background=40.0)
    img = np.clip(img.astype(int) + rng.integers(-3, 4, img.shape), 0, 127).astype(np.uint8)
    model = oracle.create_model(tmpl, 10, 20, 1, 45.0)
    base = oracle.score_map(oracle.search_fields(img, 1, 10)[0], model.points[0], 8, 45.0)
    off = oracle.score_map(oracle.search_fields(img + 100, 1, 10)[0], model.points[0], 8, 45.0)
    assert np.array_equal(base, off)
    gain = oracle.score_map(oracle.search_fields(2 * img, 1, 20)[0], model.points[0], 8, 45.0)
    assert np.array_equal(base, gain)


def test_occlusion_proportional():
    """Zeroing the search gradients under k model points (and their windows)
    lowers M from 1 by exactly k/n; the ring of the part is one such group."""
    rng = np.random.default_rng(12)
    spec = synth.PartSpec(width=40, height=40)
    spec.fill.append(("rect", 5.0, 5.0, 17.0, 35.0))     # left bar
    spec.fill.append(("circle", 29.0, 20.0, 6.0))         # separate disc
    tmpl = synth.render_template(spec)
    model = oracle.create_model(tmpl, 30, 60, 1, 90.0)
    img = synth.paste_scene(spec, (80, 80), [(40, 40, 0.0)])
    f = oracle.search_fields(img, 1, 30)[0]
    tx, ty, _, _ = model.points[0]
    n = len(tx)
    rot = oracle.rotate_points(model.points[0], 0, 90.0)
    for nb in (1, 3):
        assert oracle.score_pose(f, rot, 40, 40, nb, 0) == pytest.approx(1.0, abs=1e-12)
    # bar edge pixels have tx <= -2, disc edge pixels tx >= 2: the zeroed 3x3
    # windows of the disc points (tx >= 1) never reach a bar point's window
    disc = tx >= 0
    assert tx[~disc].max() <= -2 and tx[disc].min() >= 2
    k = int(disc.sum())
    assert 0 < k < n
    g = f.copy()
    for x, y in zip(tx[disc] + 40, ty[disc] + 40):
        g[y - 1:y + 2, x - 1:x + 2] = 0.0
    for nb in (1, 3):
        assert oracle.score_pose(g, rot, 40, 40, nb, 0) == pytest.approx((n - k) / n, abs=1e-12)


# ---------------------------------------------------------------------------
# candidates, refinement shifts, NMS
# ---------------------------------------------------------------------------

def test_candidates_golden(golden_dir):
    for c in _golden(golden_dir, "candidates.json")["cases"]:
        ck, cy, cx, cs = oracle.candidates(np.array(c["map"], np.float64), c["min_score"], c["K"])
        got = [[int(a), int(b), int(d), float(e)] for a, b, d, e in zip(ck, cy, cx, cs)]
        assert got == c["expect"]


def _brute_candidates(smap, min_score, K):
    nth, gh, gw = smap.shape
    out = []
    for k in range(nth):
        for y in range(gh):
            for x in range(gw):
                s = smap[k, y, x]
                if s < min_score:
                    continue
                key = (k, y, x)
                ok = True
                for dk in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            k2 = (k + dk) % nth
                            y2, x2 = y + dy, x + dx
                            if not (0 <= y2 < gh and 0 <= x2 < gw) or (k2, y2, x2) == key:
                                continue
                            s2 = smap[k2, y2, x2]
                            if not (s > s2 or (s == s2 and key < (k2, y2, x2))):
                                ok = False
                if ok:
                    out.append((-s, key))
    out.sort()
    return [(k, y, x, -s) for s, (k, y, x) in out[:K]]


def test_candidates_brute_force_with_ties():
    rng = np.random.default_rng(4)
    for trial in range(20):
        smap = rng.integers(0, 6, (int(rng.integers(1, 6)), 7, 9)).astype(np.float64) / 5.0
        ck, cy, cx, cs = oracle.candidates(smap, 0.4, 12)
        got = list(zip(ck.tolist(), cy.tolist(), cx.tolist(), cs.tolist()))
        assert got == _brute_candidates(smap, 0.4, 12)


def test_nms_golden(golden_dir):
    g = _golden(golden_dir, "nms.json")
    d = np.array(g["dets"])
    keep = oracle.nms(d[:, 0].astype(np.int32), d[:, 1].astype(np.int32), d[:, 2].astype(np.int32), d[:, 3],
                      100, 100, g["min_side"], 10)
    assert keep.tolist() == g["keep"]


def test_detect_config1_finds_ground_truth():
    tm, sc, truth = synth.config1_scene()
    model = oracle.create_model(tm, 30, 60, 3, 1.0)
    det = oracle.detect(model, sc, oracle.DetectParams(min_score=0.7))
    assert len(det) >= 3
    for gx, gy, gth in truth:
        best = min(det[:3], key=lambda d: math.hypot(d[0] - gx, d[1] - gy))
        assert math.hypot(best[0] - gx, best[1] - gy) <= 1.5
        dth = abs((best[2] - gth + 180) % 360 - 180)
        assert dth <= 4.0
        assert best[3] > 0.9

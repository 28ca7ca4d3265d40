"""The premise of the edge-presence bound, checked against the FP64 oracle.

The GPU scorers skip a pose when too few of its points can vote (the bound
is not in the paper; it follows from Eq. (1) with the neighbouring search):
  * a point's vote is 0 when no pixel of its 3x3 window is an edge pixel
    (the unit field is (0, 0) there), and at most 1 otherwise;
  * with polarity 0, an edge pixel whose unit vector lies in the quadrant
    opposite the point's rotated direction gives a dot product <= 0, so it
    cannot raise the vote above 0 either; quadrants are decided by signs
    alone, so this also holds for dot products rounded in FP32.
Hence n M <= E, E = the number of points whose window holds an edge pixel
not in the opposite quadrant (polarity 1: any edge pixel).  These tests
count E by brute force and compare it with the oracle's score at many
poses, instances included, where the bound is nearly tight; using the
wrong quadrant (or none of the window) makes them fail.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _quadrant(x, y):
    # [0, 90) -> 0, [90, 180) -> 1, [180, 270) -> 2, [270, 360) -> 3, by signs
    if y > 0:
        return 0 if x > 0 else 1
    if y < 0:
        return 2 if x < 0 else 3
    return 0 if x > 0 else 2


def _edge_count(field, rot, ux, uy, polarity):
    h, w = field.shape[:2]
    ox, oy, px, py = rot
    e = 0
    for i in range(len(ox)):
        opp = (_quadrant(px[i], py[i]) + 2) & 3
        hit = False
        for b in (-1, 0, 1):
            for a in (-1, 0, 1):
                x, y = ux + ox[i] + a, uy + oy[i] + b
                if 0 <= x < w and 0 <= y < h:
                    v = field[y, x]
                    if (v[0] != 0 or v[1] != 0) and (polarity or _quadrant(v[0], v[1]) != opp):
                        hit = True
        e += hit
    return e


@pytest.fixture(scope="module")
def scene():
    tmpl, img, truth = synth.config1_scene()
    om = oracle.create_model(tmpl, 30, 60, 1, 4.0)
    field = oracle.search_fields(img, 1, 30)[0]
    return om, field, truth


@pytest.mark.parametrize("polarity", [0, 1])
def test_score_never_exceeds_edge_count(scene, polarity):
    om, field, truth = scene
    pts = om.points[0]
    n = len(pts[0])
    h, w = field.shape[:2]
    rng = np.random.default_rng(13 + polarity)
    poses = [(int(round(x)), int(round(y)), int(round(th / 4.0)) % 90) for x, y, th in truth]
    poses += [(x + dx, y + dy, (k + dk) % 90) for x, y, k in poses[:2] for dx in (-1, 0, 1) for dy in (-1, 1)
              for dk in (-1, 0, 1)]
    poses += [(int(rng.integers(0, w)), int(rng.integers(0, h)), int(rng.integers(0, 90))) for _ in range(60)]
    tight = 0
    for x, y, k in poses:
        rot = oracle.rotate_points(pts, k, 4.0)
        m = oracle.score_pose(field, rot, x, y, nbhd=3, polarity=polarity)
        e = _edge_count(field, rot, x, y, polarity)
        assert n * m <= e + 1e-9, (x, y, k, n * m, e)
        tight += n * m > 0.9 * e
    # at the instances the bound is nearly tight: almost every counted point
    # votes close to 1
    assert tight >= len(truth)


def test_opposite_quadrant_dot_is_never_positive_in_fp32():
    # every sign pattern, axis directions included, rounded in FP32
    rng = np.random.default_rng(5)
    ang = np.concatenate([rng.uniform(0, 2 * np.pi, 4000), np.arange(0, 360, 90) * np.pi / 180,
                          np.array([1e-7, np.pi / 2 - 1e-7, np.pi + 1e-7, 1.5 * np.pi - 1e-7])])
    v = np.stack([np.cos(ang), np.sin(ang)], 1).astype(np.float32)
    v[np.abs(v) < 1e-6] = np.float32(0)
    q = np.array([_quadrant(a, b) for a, b in v])
    for j in range(0, len(v), 7):
        opp = q == ((q[j] + 2) & 3)
        d = v[opp, 0] * v[j, 0] + v[opp, 1] * v[j, 1]           # FP32 products and sum
        assert d.dtype == np.float32 and (d <= 0).all()
    # and a same-quadrant pair can be positive (the test can fail)
    assert (v[q == q[0], 0] * v[0, 0] + v[q == q[0], 1] * v[0, 1] > 0).any()

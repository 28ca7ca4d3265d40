"""Pins of the oracle's affine (scaled) projection, a generalisation of Eq. (2).

A pose p = A t + u with a 2x2 matrix A (A = s R(theta) for a scaled pose):
offsets rounded as in Eq. (2), model directions carried by the inverse
transpose A^-T g.  What fixes it, independently of the oracle's own code:
  * A = R(theta_k) gives exactly the integer offsets of Eq. (2) (rotate_points)
    and its directions up to FP64 rounding; A = 2 I doubles the offsets;
  * the direction rule is the gradient of the warped image: linear ramps
    warped by a squeeze, a shear or a scale, differentiated by the oracle's own Sobel,
    point exactly where the projected model directions point (A instead of
    A^-T, or A^-1 untransposed, fails it);
  * a template enlarged 2x by pixel replication scores exactly 1 at scale 2
    (and turned a quarter turn, at scale 2 and 90 degrees), well above the
    other scales tried.
"""

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def model_pts():
    import synth
    tmpl, _, _ = synth.config1_scene()
    om = oracle.create_model(tmpl, 30, 60, 1, 1.0)
    return om.points[0]


def test_rotation_is_eq2(model_pts):
    for k in (0, 17, 90, 133, 270, 359):
        rot = oracle.rotate_points(model_pts, k, 1.0)
        aff = oracle.project_affine(model_pts, oracle.similarity(1.0, k * 1.0))
        assert np.array_equal(aff[0], rot[0]) and np.array_equal(aff[1], rot[1])
        assert np.abs(aff[2] - rot[2]).max() < 1e-15 and np.abs(aff[3] - rot[3]).max() < 1e-15


def test_integer_scale_doubles_offsets(model_pts):
    tx, ty, gx, gy = model_pts
    ox, oy, px, py = oracle.project_affine(model_pts, [[2.0, 0.0], [0.0, 2.0]])
    assert np.array_equal(ox, 2 * tx) and np.array_equal(oy, 2 * ty)
    m = np.hypot(gx, gy)
    assert np.abs(px - gx / m).max() < 1e-15 and np.abs(py - gy / m).max() < 1e-15


@pytest.mark.parametrize("A,want", [
    ([[1.0, 0.0], [0.0, 0.5]], (3, 4)),      # y squeezed by 2: I'(x, y) = I(x, 2y)
    ([[1.0, 1.0], [0.0, 1.0]], (3, -1)),     # shear: I'(x, y) = I(x - y, y)
    ([[2.0, 0.0], [0.0, 2.0]], (3, 2)),      # uniform scale keeps directions (ramp halves: 1.5, 1)
])
def test_directions_follow_the_warped_image(A, want):
    # I = 40 + 3 x + 2 y; the warped image I(A^-1 x) is again a ramp whose
    # integer coefficients are `want` (up to a positive factor); its Sobel
    # gradient, from the oracle, fixes the direction a model point must take
    yy, xx = np.mgrid[0:16, 0:16]
    Ai = np.linalg.inv(np.array(A))
    a, b = np.array([3.0, 2.0]) @ Ai            # coefficients of the warped ramp
    warped = 100 + 2 * (a * xx + b * yy)        # doubled so the uniform scale stays integer
    assert np.allclose(warped, np.round(warped))
    gx, gy = oracle.sobel(warped.astype(np.uint8))
    g_img = np.array([gx[8, 8], gy[8, 8]], float)
    assert np.allclose(g_img / np.hypot(*g_img), np.array(want) / np.hypot(*want))
    # the model point of the unwarped ramp: its Sobel gradient is (24, 16)
    base = (40 + 3 * xx + 2 * yy).astype(np.uint8)
    bgx, bgy = oracle.sobel(base)
    pts = (np.array([0], np.int32), np.array([0], np.int32), np.array([bgx[8, 8]], np.int32),
           np.array([bgy[8, 8]], np.int32))
    _, _, px, py = oracle.project_affine(pts, A)
    assert abs(px[0] - g_img[0] / np.hypot(*g_img)) < 1e-12 and abs(py[0] - g_img[1] / np.hypot(*g_img)) < 1e-12


def test_template_enlarged_twice_is_found_at_scale_two():
    tm = np.full((24, 24), 60, np.uint8)
    tm[6:18, 6:18] = 200
    tm[9:12, 9:15] = 60                          # a slot, so the part is not symmetric
    om = oracle.create_model(tm, 30, 60, 1, 1.0)
    pts = om.points[0]
    scene = np.full((80, 80), 60, np.uint8)
    scene[16:64, 16:64] = np.kron(tm, np.ones((2, 2), np.uint8))
    field = oracle.search_fields(scene, 1, 30)[0]
    # the template's reference pixel (12, 12) covers scene pixels 40..41
    best = {}
    for s in (1.0, 1.5, 2.0, 2.5):
        rot = oracle.project_affine(pts, oracle.similarity(s, 0.0))
        best[s] = max(oracle.score_pose(field, rot, x, y) for x in range(38, 44) for y in range(38, 44))
    assert abs(best[2.0] - 1.0) < 1e-12
    assert max(v for s, v in best.items() if s != 2.0) < 0.7
    # and a quarter turn of the enlarged part at scale 2 and 90 degrees
    scene90 = np.ascontiguousarray(np.rot90(scene, -1))     # turned 90 degrees with y down
    f90 = oracle.search_fields(scene90, 1, 30)[0]
    rot = oracle.project_affine(pts, oracle.similarity(2.0, 90.0))
    b90 = max(oracle.score_pose(f90, rot, x, y) for x in range(36, 46) for y in range(36, 46))
    assert abs(b90 - 1.0) < 1e-12

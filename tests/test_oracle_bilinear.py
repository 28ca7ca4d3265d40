"""Pins of the oracle's differentiable score (continuous pose) and of its
damped Gauss-Newton pose refinement.

The continuous score extends Eq. (1) to non-integer poses: Eq. (2) without
rounding and a bilinear sample of the unit search field.  It is pinned to
the integer-pose score (already pinned to the paper), to closed forms on
fields whose bilinear interpolation is exact (constant and affine fields),
to central finite differences, to 90-degree rotation of the image, and, for
the refinement, to a noise-free pasted template whose pose is known.
"""

import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def part():
    rng = np.random.default_rng(71)
    spec = synth.random_part(rng, 40, kind="part", margin=3.0)
    tmpl = synth.render_template(spec)
    return spec, tmpl, oracle.model_points(tmpl, 30, 60)


@pytest.fixture(scope="module")
def scene_field(part):
    spec, tmpl, pts = part
    img = synth.paste_scene(spec, (128, 112), [(60, 52, 23.0)])
    rng = np.random.default_rng(5)
    img = np.clip(img.astype(np.float64) + rng.normal(0, 3.0, img.shape), 0, 255).astype(np.uint8)
    return oracle.search_fields(img, 1, 30)[0]


def _unit_dirs(pts):
    gx, gy = pts[2].astype(np.float64), pts[3].astype(np.float64)
    m = np.hypot(gx, gy)
    return gx / m, gy / m


def test_integer_pose_equals_discrete_score(part, scene_field):
    # at theta in {0, 90, 180, 270} and an integer u every sample falls on a
    # pixel, so the continuous score is the neighbourhood-1 score of Eq. (1)
    _, _, pts = part
    for k, th in enumerate([0.0, 90.0, 180.0, 270.0]):
        rot = oracle.rotate_points(pts, k, 90.0)
        for ux, uy in [(60, 52), (61, 50), (30, 80), (2, 3)]:
            ref = oracle.score_pose(scene_field, rot, ux, uy, nbhd=1)
            got = oracle.score_bilinear(scene_field, pts, ux, uy, th)
            assert abs(got - ref) < 1e-12, (th, ux, uy)
            ref1 = oracle.score_pose(scene_field, rot, ux, uy, nbhd=1, polarity=1)
            got1 = oracle.score_bilinear(scene_field, pts, ux, uy, th, polarity=1)
            assert abs(got1 - ref1) < 1e-12


def test_constant_field_closed_form(part):
    # w_hat = v everywhere => M_c = (1/n) sum (R g_i/|g_i|) . v, independent
    # of u; dM/dtheta = (1/n) sum (R' g_i/|g_i|) . v * pi/180
    _, _, pts = part
    v = np.array([0.6, -0.8])
    field = np.zeros((200, 200, 2))
    field[...] = v
    ux, uy = _unit_dirs(pts)
    for th in [0.0, 17.3, 123.4, 271.9]:
        r = math.radians(th)
        c, s = math.cos(r), math.sin(r)
        # v turned back by -theta, dotted with the unturned directions
        vb = np.array([c * v[0] + s * v[1], -s * v[0] + c * v[1]])
        want = np.mean(ux * vb[0] + uy * vb[1])
        dvb = np.array([-s * v[0] + c * v[1], -c * v[0] - s * v[1]])
        dwant = np.mean(ux * dvb[0] + uy * dvb[1]) * math.pi / 180
        got, o = oracle.score_bilinear(field, pts, 100.3, 99.6, th, want=("grad",))
        assert abs(got - want) < 1e-13
        assert abs(o["grad"][0]) < 1e-13 and abs(o["grad"][1]) < 1e-13
        assert abs(o["grad"][2] - dwant) < 1e-13


def test_affine_field_closed_form(part):
    # an affine field is reproduced exactly by bilinear interpolation, so the
    # score is a closed-form function of the pose.  Different slopes in x
    # and y catch swapped interpolation weights; the theta derivative has
    # both the turned-direction and the moved-sample parts.
    _, _, pts = part
    H, W = 220, 240
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    A = np.array([[0.003, -0.002], [0.0015, 0.004]])   # field = A @ (x, y) + b
    b = np.array([-0.1, 0.2])
    field = np.stack([A[0, 0] * xs + A[0, 1] * ys + b[0], A[1, 0] * xs + A[1, 1] * ys + b[1]], axis=-1)
    ux, uy = _unit_dirs(pts)
    tx, ty = pts[0].astype(np.float64), pts[1].astype(np.float64)
    for (x, y, th) in [(120.25, 101.75, 0.0), (118.6, 99.1, 33.3), (121.9, 110.45, 250.8)]:
        r = math.radians(th)
        c, s = math.cos(r), math.sin(r)
        px, py = c * tx - s * ty + x, s * tx + c * ty + y
        dx, dy = c * ux - s * uy, s * ux + c * uy
        wx = A[0, 0] * px + A[0, 1] * py + b[0]
        wy = A[1, 0] * px + A[1, 1] * py + b[1]
        want = np.mean(dx * wx + dy * wy)
        gx_ = np.mean(dx * A[0, 0] + dy * A[1, 0])
        gy_ = np.mean(dx * A[0, 1] + dy * A[1, 1])
        # theta: d/dtheta of d . (A p + b), p = R t + u
        ddx, ddy = -s * ux - c * uy, c * ux - s * uy
        dpx, dpy = -s * tx - c * ty, c * tx - s * ty
        gt_ = np.mean(ddx * wx + ddy * wy + dx * (A[0, 0] * dpx + A[0, 1] * dpy)
                      + dy * (A[1, 0] * dpx + A[1, 1] * dpy)) * math.pi / 180
        got, o = oracle.score_bilinear(field, pts, x, y, th, want=("grad",))
        assert abs(got - want) < 1e-12
        np.testing.assert_allclose(o["grad"], [gx_, gy_, gt_], rtol=0, atol=1e-12)


def test_gradient_matches_central_differences(part, scene_field):
    # h = 1e-6: poses with no sample within 4h of a cell border, so every
    # coordinate stays in one cell; the score is then bilinear in (x, y)
    _, _, pts = part
    rng = np.random.default_rng(3)
    h = 1e-6
    checked = 0
    for _ in range(40):
        pose = (60 + rng.uniform(-1.5, 1.5), 52 + rng.uniform(-1.5, 1.5), 23 + rng.uniform(-1.5, 1.5))
        if oracle.bilinear_border_mask(pts, *pose, 4 * h).any():
            continue
        for pol in (0, 1):
            _, o = oracle.score_bilinear(scene_field, pts, *pose, polarity=pol, want=("grad",))
            for j in range(3):
                a, b = list(pose), list(pose)
                a[j] += h
                b[j] -= h
                fd = (oracle.score_bilinear(scene_field, pts, *a, polarity=pol)
                      - oracle.score_bilinear(scene_field, pts, *b, polarity=pol)) / (2 * h)
                assert abs(fd - o["grad"][j]) < 2e-7, (pose, pol, j, fd, o["grad"][j])
        checked += 1
    assert checked >= 20


def test_gradient_central_differences_h1e3(part, scene_field):
    # h = 1e-3 px / deg over the points whose sample stays inside one cell
    # for every perturbation (the others' one-sided derivative may jump)
    _, _, pts = part
    rng = np.random.default_rng(4)
    h = 1e-3
    rmax = float(np.max(np.hypot(pts[0], pts[1])))
    eps = max(h, rmax * math.radians(h)) * 1.5
    for _ in range(10):
        pose = (60 + rng.uniform(-1.5, 1.5), 52 + rng.uniform(-1.5, 1.5), 23 + rng.uniform(-1.5, 1.5))
        keep = ~oracle.bilinear_border_mask(pts, *pose, eps)
        sub = tuple(a[keep] for a in pts)
        assert keep.sum() > 0.8 * len(keep)
        _, o = oracle.score_bilinear(scene_field, sub, *pose, want=("grad",))
        for j in range(3):
            a, b = list(pose), list(pose)
            a[j] += h
            b[j] -= h
            fd = (oracle.score_bilinear(scene_field, sub, *a) - oracle.score_bilinear(scene_field, sub, *b)) / (2 * h)
            assert abs(fd - o["grad"][j]) < 1e-6, (pose, j)


def test_normal_equations_definition(part, scene_field):
    # J^T J is positive semi-definite and J^T r = grad - (1/n) sum J_i term_i
    # reduces to grad where every term is 0 (a field of zeros gives 0 for all)
    _, _, pts = part
    _, o = oracle.score_bilinear(scene_field, pts, 60.3, 51.8, 22.6, want=("grad", "jtj", "jtr"))
    a = o["jtj"]
    M = np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])
    assert np.linalg.eigvalsh(M).min() > -1e-15
    zero = np.zeros_like(scene_field)
    s0, o0 = oracle.score_bilinear(zero, pts, 60.3, 51.8, 22.6, want=("grad", "jtj", "jtr"))
    assert s0 == 0.0 and not o0["grad"].any() and not o0["jtj"].any() and not o0["jtr"].any()


def test_quarter_turn_of_image(part, scene_field):
    # turning the image (and its gradient field) by 90 degrees and the pose
    # with it leaves the continuous score unchanged
    _, _, pts = part
    H, W = scene_field.shape[:2]
    # image I'(x', y') = I(y', W-1-x')... use numpy rot90 (counter-clockwise
    # in array view = clockwise turn of x-right/y-down coordinates)
    f2 = np.rot90(scene_field, k=1, axes=(0, 1)).copy()
    # a point (x, y) of the old image is at (y, W-1-x) of the new one; the
    # field vector (wx, wy) becomes (wy, -wx) there
    f2 = np.stack([f2[..., 1], -f2[..., 0]], axis=-1)
    for pose in [(60.4, 52.3, 23.7), (58.9, 50.2, 21.1)]:
        x, y, th = pose
        s1 = oracle.score_bilinear(scene_field, pts, x, y, th)
        s2 = oracle.score_bilinear(f2, pts, y, W - 1 - x, th - 90.0)
        assert abs(s1 - s2) < 1e-12


def test_refine_converges_on_pasted_template(part):
    # noise-free template pasted at an integer pose with theta = 0: the
    # maximum M_c = 1 is at that pose; the refinement reaches it from a
    # perturbed start and never lowers the score
    spec, tmpl, pts = part
    img = synth.paste_scene(spec, (120, 100), [(57, 49, 0.0)])
    field = oracle.search_fields(img, 1, 30)[0]
    assert abs(oracle.score_bilinear(field, pts, 57, 49, 0.0) - 1.0) < 1e-12
    rng = np.random.default_rng(8)
    for _ in range(6):
        init = (57 + rng.uniform(-0.8, 0.8), 49 + rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8))
        s0 = oracle.score_bilinear(field, pts, *init)
        p, s = oracle.refine_gn(field, pts, init, iterations=30)
        assert s >= s0
        assert abs(s - oracle.score_bilinear(field, pts, *p)) < 1e-15
        assert np.abs(p - np.array([57, 49, 0.0])).max() < 0.02, (init, p)
        assert s > 0.98


def test_refine_zero_iterations_is_identity(part, scene_field):
    _, _, pts = part
    p, s = oracle.refine_gn(scene_field, pts, (60.2, 52.1, 23.3), iterations=0)
    assert list(p) == [60.2, 52.1, 23.3]
    assert s == oracle.score_bilinear(scene_field, pts, 60.2, 52.1, 23.3)


def test_refine_step_is_the_damped_normal_equation_solution(part):
    # one iteration moves to p + d with (J^T J + 1e-3 diag(J^T J) + 1e-9 I) d
    # = J^T r solved by LAPACK (d scaled to max |d_j| <= 1), when M_c rises
    spec, tmpl, pts = part
    img = synth.paste_scene(spec, (120, 100), [(57, 49, 0.0)])
    field = oracle.search_fields(img, 1, 30)[0]
    rng = np.random.default_rng(12)
    moved = clamped = 0
    for r in [0.6] * 8 + [2.5] * 8:
        p0 = np.array([57 + rng.uniform(-r, r), 49 + rng.uniform(-r, r), rng.uniform(-r, r)])
        s0, o = oracle.score_bilinear(field, pts, *p0, want=("jtj", "jtr"))
        a = o["jtj"]
        A = np.array([[a[0], a[1], a[2]], [a[1], a[3], a[4]], [a[2], a[4], a[5]]])
        A = A + 1e-3 * np.diag(np.diag(A)) + 1e-9 * np.eye(3)
        d = np.linalg.solve(A, o["jtr"])
        clamped += bool(np.abs(d).max() > 1.0)
        d = d / max(1.0, np.abs(d).max())
        want = p0 + d if oracle.score_bilinear(field, pts, *(p0 + d)) > s0 else p0
        p1, _ = oracle.refine_gn(field, pts, p0, iterations=1)
        np.testing.assert_allclose(p1, want, rtol=0, atol=1e-12)
        moved += bool((p1 != p0).any())
    assert moved >= 8 and clamped >= 3

"""Pins of the oracle's sub-pixel / sub-angle quadratic fit (the first
widening of the digitised pose: the peak of a 3x3x3 neighbourhood of Eq. (1)
scores).

The fit is the stationary point of the second-order Taylor model of the
scores from central differences.  Pinned against what the mathematics fixes:
- any quadratic with a negative definite Hessian and its vertex inside the
  cell is recovered exactly (every stencil, sign, index and the mixed terms);
- a separable neighbourhood gives the textbook three-point parabola vertex
  per axis;
- a vertex outside the cell is clamped to +-1/2; a saddle falls back to the
  axes that curve down; a symmetric neighbourhood gives 0;
- on a scene, the fitted pose of a translated image moves with the image,
  and the fit moves an instance's angle toward its off-grid truth.
"""

import numpy as np
import pytest

import oracle
import synth


def _grid():
    d = np.array([-1.0, 0.0, 1.0])
    dk, dy, dx = np.meshgrid(d, d, d, indexing="ij")
    return np.stack([dx.ravel(), dy.ravel(), dk.ravel()], axis=1)   # (27, 3) in (x, y, k) order


def _quadratic(H, v, c):
    P = _grid() - v
    return c + 0.5 * np.einsum("ni,ij,nj->n", P, H, P)


@pytest.mark.parametrize("seed", range(12))
def test_exact_on_quadratics(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3))
    H = -(A @ A.T + 0.2 * np.eye(3))                     # negative definite, full mixed terms
    v = rng.uniform(-0.45, 0.45, size=3)
    s = _quadratic(H, v, rng.uniform(0.5, 1.0))
    assert np.allclose(oracle.subpixel_fit(s), v, atol=1e-12)


def test_separable_is_three_point_parabola():
    rng = np.random.default_rng(5)
    P = _grid()
    a = rng.uniform(0.05, 0.4, size=3)
    v = rng.uniform(-0.4, 0.4, size=3)
    s = 0.9 - (a * (P - v) ** 2).sum(axis=1)
    S = s.reshape(3, 3, 3)   # [k][y][x]
    lines = (S[1, 1, :], S[1, :, 1], S[:, 1, 1])
    want = [(m[0] - m[2]) / (2.0 * (m[0] - 2.0 * m[1] + m[2])) for m in lines]
    assert np.allclose(oracle.subpixel_fit(s), want, atol=1e-12)
    assert np.allclose(want, v, atol=1e-12)


def test_symmetric_and_clamped():
    P = _grid()
    s = 1.0 - 0.1 * (P ** 2).sum(axis=1)
    assert np.allclose(oracle.subpixel_fit(s), 0.0, atol=1e-15)
    far = _quadratic(-np.diag([0.2, 0.3, 0.1]), np.array([0.8, -1.7, 0.3]), 1.0)
    assert np.allclose(oracle.subpixel_fit(far), [0.5, -0.5, 0.3], atol=1e-12)


def test_saddle_falls_back_to_the_axes_that_curve_down():
    H = np.diag([-0.3, 0.2, -0.1])
    v = np.array([0.2, 0.1, -0.3])
    s = _quadratic(H, v, 1.0)
    # x and k curve down: their own parabola vertices; y curves up: 0
    assert np.allclose(oracle.subpixel_fit(s), [0.2, 0.0, -0.3], atol=1e-12)


def test_translation_moves_the_fit_with_the_image():
    tm, sc, gts = synth.config1_scene()
    om = oracle.create_model(tm, 30, 60, 1, 4.0)
    x, y, th = gts[0]
    k = int(round(th / 4.0)) % 90
    pts = om.points[0]
    f = oracle.search_fields(sc, 1, 30)[0]
    shifted = np.zeros_like(sc) + sc[0, 0]
    shifted[3:, 5:] = sc[:-3, :-5]
    g = oracle.search_fields(shifted, 1, 30)[0]
    a = oracle.subpixel_poses(f, pts, [(k, y, x)], 90, 4.0)[0]
    b = oracle.subpixel_poses(g, pts, [(k, y + 3, x + 5)], 90, 4.0)[0]
    assert np.allclose(b[:3], a[:3] + [5.0, 3.0, 0.0], atol=1e-12)


def test_fit_moves_angle_toward_off_grid_truth():
    # config-2 instances sit on a 0.5 degree grid; at a 1 degree angle step
    # the integer search is up to 0.5 degree off, the fit must not be worse
    # on average and must be better where the truth is off the grid
    W, H = 640, 512
    errs_int, errs_fit = [], []
    spec = None
    for seed in range(4):
        tm, sc, gts, spec = synth.config2_scene(seed=5000 + seed, W=W, H=H, side=120, spec=spec, n_inst=2)
        om = oracle.create_model(tm, 30, 60, 1, 1.0)
        f = oracle.search_fields(sc, 1, 30)[0]
        for (x, y, th) in gts:
            k = int(round(th)) % 360
            p = oracle.subpixel_poses(f, om.points[0], [(k, int(round(y)), int(round(x)))], 360, 1.0)[0]
            dint = abs(((k - th) + 180.0) % 360.0 - 180.0)
            dfit = abs(((p[2] - th) + 180.0) % 360.0 - 180.0)
            if dint > 0.25:
                errs_int.append(dint)
                errs_fit.append(dfit)
    assert len(errs_int) >= 2
    assert np.mean(errs_fit) < np.mean(errs_int)


def test_climb_picks_the_strictly_best_neighbour():
    s = np.zeros(27)
    s[13] = 1.0
    assert oracle.climb27(s) == 13                 # the centre is the best
    s[4] = 1.0
    assert oracle.climb27(s) == 13                 # a tie keeps the centre
    s[22] = 1.5
    s[5] = 1.5
    assert oracle.climb27(s) == 5                  # first of the equal best
    assert oracle.climb27(np.arange(27.0)) == 26


def test_climb_reaches_the_same_peak_from_a_neighbouring_start():
    tm, sc, gts = synth.config1_scene()
    om = oracle.create_model(tm, 30, 60, 1, 4.0)
    f = oracle.search_fields(sc, 1, 30)[0]
    x, y, th = gts[0]
    k = int(round(th / 4.0)) % 90
    a = oracle.subpixel_poses(f, om.points[0], [(k, y, x)], 90, 4.0)[0]
    b = oracle.subpixel_poses(f, om.points[0], [(k, y + 1, x - 1)], 90, 4.0)[0]
    c = oracle.subpixel_poses(f, om.points[0], [(k, y + 1, x - 1)], 90, 4.0, max_moves=0)[0]
    assert np.allclose(a, b, atol=1e-12)
    assert not np.allclose(c[:2], a[:2], atol=1e-6)   # without moves the fit stays in the start's cell

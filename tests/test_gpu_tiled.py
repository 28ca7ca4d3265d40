"""GPU parity of the tiled exhaustive scorer (TMA window, register blocking).

Checked against the FP64 oracle (1e-5 absolute) and against the generic
one-thread-per-pose kernel on: several CTA tilings and angle groupings,
neighbourhood 1 and 3, both polarities, early termination (exact-safe),
ragged image sizes (odd widths, partial warp tiles), images smaller than
one warp tile, and the full 160x128 top level of a 1280x1024 search.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    yield
    sam.set_score_kernel(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _map(model, level, img, kernel, cfg=(2, 1, 9, 8), nbhd=3, min_score=0.0, early=0):
    h, w = img.shape
    sam.set_score_kernel(kernel, *cfg)
    wp = sam.field_pitch(w, sam.LAYOUT_PAIRS)
    f = torch.zeros((h, wp, 2), dtype=torch.float32, device="cuda")
    sam.gradient(_dev(img), model.params.low, sam.FP32, f, layout=sam.LAYOUT_PAIRS)
    nth = model.num_angles(level)
    out = torch.full((nth, h, w), float("nan"), dtype=torch.float32, device="cuda")
    sam.score_map(model, level, f, w, h, sam.FP32, out, 1, 1, nbhd, min_score, early, layout=sam.LAYOUT_PAIRS)
    torch.cuda.synchronize()
    assert sam.take_device_error() == 0
    return out.cpu().numpy()


def _oracle_map(om, level, img, nbhd=3):
    f = oracle.search_fields(img, 1, om.low)[0]
    return oracle.score_map(f, om.points[level], om.ntheta(level), om.dtheta(level), nbhd=nbhd,
                            polarity=om.polarity)


def test_pairs_layout_gradient_matches_pixel_layout():
    rng = np.random.default_rng(1)
    for h, w in [(61, 77), (128, 160), (3, 5), (40, 2)]:
        img = rng.integers(0, 256, (h, w)).astype(np.uint8)
        fa = torch.empty((h, w, 2), dtype=torch.float32, device="cuda")
        sam.gradient(_dev(img), 10, sam.FP32, fa)
        wp = sam.field_pitch(w, sam.LAYOUT_PAIRS)
        fb = torch.full((h, wp * 2), 7.0, dtype=torch.float32, device="cuda")
        sam.gradient(_dev(img), 10, sam.FP32, fb, layout=sam.LAYOUT_PAIRS)
        torch.cuda.synchronize()
        a = fa.cpu().numpy()
        b = fb.cpu().numpy().reshape(h, wp // 2, 4)
        wx = b[:, :, 0:2].reshape(h, wp)
        wy = b[:, :, 2:4].reshape(h, wp)
        assert np.array_equal(wx[:, :w], a[..., 0]) and np.array_equal(wy[:, :w], a[..., 1])
        if wp > w:
            assert np.all(wx[:, w:] == 0) and np.all(wy[:, w:] == 0)


@pytest.mark.parametrize("cfg", [(2, 1, 9, 8), (1, 1, 1, 4), (3, 2, 45, 8), (1, 4, 7, 4), (2, 2, 90, 8),
                                 (2, 1, 9, 8, 10), (1, 1, 3, 4, 10), (2, 2, 5, 8, 10), (1, 2, 45, 4, 10),
                                 (2, 2, 0, 4), (4, 1, 0, 4), (1, 4, 0, 4), (2, 4, 0, 8), (4, 2, 0, 8)])
def test_tiled_matches_oracle_config1_top(cfg):
    # tg = 0: the chunked kernel; a fifth value: pose columns per thread
    tm, sc, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, 3, 1.0)
    om = oracle.create_model(tm, 30, 60, 3, 1.0)
    top = oracle.pyramid(sc, 3)[2]
    got = _map(m, 2, top, 2, cfg)
    ref = _oracle_map(om, 2, top)
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("nbhd,polarity", [(1, 0), (3, 1), (1, 1)])
def test_tiled_neighbourhood_and_polarity(nbhd, polarity):
    tm, sc, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, 3, 1.0, polarity)
    om = oracle.create_model(tm, 30, 60, 3, 1.0, polarity)
    top = oracle.pyramid(sc, 3)[2]
    got = _map(m, 2, top, 2, nbhd=nbhd)
    ref = _oracle_map(om, 2, top, nbhd=nbhd)
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("nbhd,polarity", [(1, 0), (3, 1), (1, 1), (3, 0)])
def test_persistent_early_termination_exact_safe(nbhd, polarity):
    # early termination runs the persistent form (edge-presence bound with a
    # plane per quadrant for polarity 0, one plane for polarity 1; surviving
    # slices scored as tasks split over the warps): every pruned pose is below
    # min_score in the oracle, every other pose matches it, none at or above
    # min_score is pruned
    tm, sc, _, _ = synth.config2_scene(seed=4321)
    m = sam.Model(tm, 30, 60, 4, 1.0, polarity)
    om = oracle.create_model(tm, 30, 60, 4, 1.0, polarity)
    top = oracle.pyramid(sc, 4)[3]
    ref = _oracle_map(om, 3, top, nbhd=nbhd)
    for ms, cfg in ((0.5, (2, 1, 11, 4, 10)), (0.7, (1, 2, 5, 8, 6))):
        got = _map(m, 3, top, 2, cfg, nbhd=nbhd, min_score=ms, early=1)
        pruned = np.isneginf(got)
        assert pruned.any()
        assert np.all(ref[pruned] < ms)
        assert not np.any(pruned & (ref >= ms))
        assert np.max(np.abs(got[~pruned] - ref[~pruned])) < TOL


@pytest.mark.parametrize("h,w", [(61, 77), (33, 49), (7, 5), (97, 145), (32, 48), (1, 1)])
def test_tiled_ragged_sizes_match_generic_and_oracle(h, w):
    tm, sc, _ = synth.tiny_case(h * 1000 + w, size=max(h, w, 24), tsize=11)
    img = np.ascontiguousarray(sc[:h, :w])
    m = sam.Model(tm, 10, 20, 1, 15.0)
    om = oracle.create_model(tm, 10, 20, 1, 15.0)
    got = _map(m, 0, img, 2, (1, 1, 5, 4))
    gen = _map(m, 0, img, 1)
    chk = _map(m, 0, img, 2, (2, 2, 0, 4))
    wide = _map(m, 0, img, 2, (1, 2, 3, 8, 10))
    ref = _oracle_map(om, 0, img)
    assert np.max(np.abs(got - ref)) < TOL
    assert np.max(np.abs(got - gen)) < TOL
    assert np.max(np.abs(chk - ref)) < TOL
    assert np.max(np.abs(wide - ref)) < TOL


def test_tiled_early_termination_exact_safe():
    tm, sc, _, _ = synth.config2_scene()
    m = sam.Model(tm, 30, 60, 4, 1.0)
    om = oracle.create_model(tm, 30, 60, 4, 1.0)
    top = oracle.pyramid(sc, 4)[3]
    ref = _oracle_map(om, 3, top)
    full = _map(m, 3, top, 2)
    assert np.max(np.abs(full - ref)) < TOL
    for ms, cfg in ((0.5, (2, 1, 9, 8)), (0.6, (2, 1, 9, 8)), (0.8, (2, 1, 9, 8)), (0.6, (2, 2, 0, 4)),
                    (0.8, (2, 4, 0, 8)), (0.6, (1, 1, 3, 8, 10)), (0.8, (2, 1, 5, 4, 10))):
        got = _map(m, 3, top, 2, cfg, min_score=ms, early=1)
        pruned = np.isneginf(got)
        assert np.all(ref[pruned] < ms)
        assert np.max(np.abs(got[~pruned] - ref[~pruned])) < TOL
        # every pose at or above min_score survives
        assert not np.any(pruned & (ref >= ms))


def test_tiled_batch_detection_matches_generic():
    imgs, tm, spec = [], None, None
    for i in range(4):
        t, sc, _, spec = synth.config2_scene(seed=7000 + i, spec=spec)
        tm = t if tm is None else tm
        imgs.append(sc)
    m = sam.Model(tm, 30, 60, 4, 1.0)
    p = sam.default_detect_params(min_score=0.6)
    batch = _dev(np.stack(imgs))
    sam.set_score_kernel(2)
    tiled = sam.detect_batch(m, batch, p)
    sam.set_score_kernel(1)
    generic = sam.detect_batch(m, batch, p)
    sam.set_score_kernel(0)
    for a, b in zip(tiled, generic):
        assert [(d["x"], d["y"], d["k"]) for d in a] == [(d["x"], d["y"], d["k"]) for d in b]
        assert all(abs(x["score"] - y["score"]) < TOL for x, y in zip(a, b))


def test_autotune_picks_a_tiling_and_keeps_results():
    imgs, tm, spec = [], None, None
    for i in range(2):
        t, sc, _, spec = synth.config2_scene(seed=7100 + i, spec=spec, W=640, H=512)
        tm = t if tm is None else tm
        imgs.append(sc)
    m = sam.Model(tm, 30, 60, 3, 1.0)
    p = sam.default_detect_params(min_score=0.6)
    batch = _dev(np.stack(imgs))
    sam.set_score_kernel(0)
    before = sam.detect_batch(m, batch, p)
    res = sam.autotune(m, batch, p)
    assert len(res) >= 10 and all(ms > 0 for _, ms in res)
    assert sam.model_tiling(m) == res[0][0]
    after = sam.detect_batch(m, batch, p)
    assert [[(d["x"], d["y"], d["k"]) for d in a] for a in after] == \
        [[(d["x"], d["y"], d["k"]) for d in b] for b in before]


@pytest.mark.parametrize("cfg", [(2, 1, 9, 8), (1, 1, 3, 8), (2, 2, 0, 4), (1, 1, 3, 4, 10)])
def test_executed_pose_point_counter(cfg):
    # without early termination every pose inside the map evaluates every
    # point: the counter equals the nominal count; with it, fewer
    tm, sc, _, _ = synth.config2_scene()
    m = sam.Model(tm, 30, 60, 4, 1.0)
    top = oracle.pyramid(sc, 4)[3]
    h, w = top.shape
    nominal = m.num_angles(3) * h * w * m.num_points(3)
    sam.executed_pose_points(reset=True)
    _map(m, 3, top, 2, cfg, early=0)
    assert sam.executed_pose_points(reset=True) == nominal
    _map(m, 3, top, 2, cfg, min_score=0.6, early=1)
    ex = sam.executed_pose_points(reset=True)
    assert 0 < ex < nominal


def test_tiled_longest_single_window_sum_matches_oracle():
    # the largest part whose rotated extent (with the edge bitmaps) still
    # fits one staged window at the smallest tiling (one angle per CTA, 4
    # warps): a 104-pixel part of 1077 points, every pose's vote sum taken
    # serially over all its points in FP32, held to 1e-5 of the FP64 oracle
    # (the worst-case rounding bound is 2^-25 n = 3.2e-5; the errors of
    # random sign stay far below it)
    rng = np.random.default_rng(77)
    spec = synth.random_part(rng, 104, kind="part", margin=3.0)
    tm = synth.render_template(spec)
    img = synth.paste_scene(spec, (160, 128), [(80.0, 64.0, 30.0)])
    img = np.clip(img.astype(np.int32) + rng.integers(-6, 7, img.shape), 0, 255).astype(np.uint8)
    model = sam.Model(tm, 30, 60, 1, 45.0)
    om = oracle.create_model(tm, 30, 60, 1, 45.0)
    assert model.num_points(0) >= 1000
    got = _map(model, 0, img, 2, cfg=(1, 1, 1, 4, 6))
    generic = _map(model, 0, img, 1)
    ref = _oracle_map(om, 0, img)
    assert np.max(np.abs(got - ref)) < TOL
    assert np.max(np.abs(generic - ref)) < TOL


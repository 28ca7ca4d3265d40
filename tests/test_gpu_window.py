"""GPU parity of windowed exhaustive scoring and of the chunked scorer.

A pose window (translation box x angle range) must reproduce the matching
slice of the full score map bit for bit (same kernel arithmetic, every pose
evaluated).  Templates too large for one staged window (400-512 pixels at
full resolution, ~4000-6000 edge points) are scored by the chunked kernel;
its scores are checked against the FP64 oracle on sampled poses and against
the generic kernel on a whole map, with early termination exact-safe, in
FP32 and in the 16-bit forms with FP32 rescoring.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

TOL = 1e-5
PREC_DTYPE = {sam.FP32: torch.float32, sam.FP16: torch.float16, sam.BF16: torch.bfloat16}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    sam.set_score_kernel(0)
    yield
    sam.set_score_kernel(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pairs_field(img, low, prec):
    h, w = img.shape
    wp = sam.field_pitch(w, sam.LAYOUT_PAIRS)
    f = torch.zeros((h, wp, 2), dtype=PREC_DTYPE[prec], device="cuda")
    sam.gradient(_dev(img), low, prec, f, layout=sam.LAYOUT_PAIRS)
    return f


def _pixel_field32(img, low):
    h, w = img.shape
    f = torch.zeros((h, w, 2), dtype=torch.float32, device="cuda")
    sam.gradient(_dev(img), low, sam.FP32, f, layout=sam.LAYOUT_PIXEL)
    return f


def _window(model, f, img, prec, win, early=0, min_score=0.0, field32=None, scratch=None, nbhd=3):
    h, w = img.shape
    x0, y0, gw, gh, k0, nk = win
    out = torch.full((nk, gh, gw), float("nan"), dtype=torch.float32, device="cuda")
    sam.score_window(model, 0, f, w, h, prec, x0, y0, gw, gh, k0, nk, out, nbhd=nbhd, min_score=min_score,
                     early=early, field32=field32, scratch=scratch)
    torch.cuda.synchronize()
    assert sam.take_device_error() == 0
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def small_case():
    tmpl, img, _ = synth.config1_scene()
    model = sam.Model(tmpl, 30, 60, 1, 4.0)
    return tmpl, img, model


@pytest.mark.parametrize("win", [(0, 0, 320, 240, 0, 90), (37, 11, 101, 67, 5, 13), (1, 2, 3, 5, 89, 1),
                                 (200, 100, 120, 140, 40, 50)])
def test_window_equals_full_map_slice(small_case, win):
    tmpl, img, model = small_case
    h, w = img.shape
    f = _pairs_field(img, 30, sam.FP32)
    full = torch.full((90, h, w), float("nan"), dtype=torch.float32, device="cuda")
    sam.score_map(model, 0, f, w, h, sam.FP32, full, 1, 1, 3, 0.0, 0, layout=sam.LAYOUT_PAIRS)
    full = full.cpu().numpy()
    x0, y0, gw, gh, k0, nk = win
    got = _window(model, f, img, sam.FP32, win)
    assert np.array_equal(got, full[k0:k0 + nk, y0:y0 + gh, x0:x0 + gw])


def test_window_rejects_bad_ranges(small_case):
    tmpl, img, model = small_case
    h, w = img.shape
    f = _pairs_field(img, 30, sam.FP32)
    out = torch.empty((1, 8, 8), dtype=torch.float32, device="cuda")
    for win in [(-1, 0, 8, 8, 0, 1), (w - 7, 0, 8, 8, 0, 1), (0, h - 7, 8, 8, 0, 1), (0, 0, 8, 8, 90, 1),
                (0, 0, 8, 8, 0, 0), (0, 0, 0, 8, 0, 1)]:
        with pytest.raises(sam.SamError):
            sam.score_window(model, 0, f, w, h, sam.FP32, *win, out)


@pytest.fixture(scope="module")
def big_case():
    # a 400-pixel part at full resolution: its rotated extent (~566 px)
    # exceeds one window, so the chunked kernel scores it
    rng = np.random.default_rng(31)
    spec = synth.random_part(rng, 400, kind="part", margin=6.0)
    tmpl, img, poses, _ = synth.config2_scene(seed=77, W=1024, H=768, side=400, spec=spec, n_inst=2)
    model = sam.Model(tmpl, 30, 60, 1, 0.5)
    om = oracle.create_model(tmpl, 30, 60, 1, 0.5)
    return tmpl, img, poses, model, om


def test_chunked_matches_oracle_on_sampled_poses(big_case):
    tmpl, img, poses, model, om = big_case
    h, w = img.shape
    assert om.points[0][0].size > 3000
    f = _pairs_field(img, 30, sam.FP32)
    ofield = oracle.search_fields(img, 1, 30)[0]
    # one angle slice over the whole image and a translation window over
    # many angles around an instance
    x, y, th = poses[0]
    k = int(round(th / 0.5)) % 720
    wins = [(0, 0, w, h, k, 1), (int(x) - 40, int(y) - 30, 96, 64, min(max(0, k - 5), 709), 11)]
    rng = np.random.default_rng(2)
    for win in wins:
        x0, y0, gw, gh, k0, nk = win
        got = _window(model, f, img, sam.FP32, win)
        assert np.isfinite(got).all()
        for _ in range(300):
            kk, yy, xx = (int(rng.integers(0, nk)), int(rng.integers(0, gh)), int(rng.integers(0, gw)))
            rot = oracle.rotate_points(om.points[0], k0 + kk, 0.5)
            ref = oracle.score_pose(ofield, rot, x0 + xx, y0 + yy, nbhd=3)
            assert abs(got[kk, yy, xx] - ref) < TOL, (win, kk, yy, xx)
        # the best pose of the instance's window is the instance
        if nk > 1:
            kk, yy, xx = np.unravel_index(np.argmax(got), got.shape)
            assert abs(x0 + xx - x) <= 1 and abs(y0 + yy - y) <= 1 and got.max() > 0.4


def test_chunked_full_map_matches_generic(big_case):
    tmpl, img, poses, model, om = big_case
    sub = np.ascontiguousarray(img[100:100 + 300, 200:200 + 400])
    h, w = sub.shape
    f = _pairs_field(sub, 30, sam.FP32)
    nth = model.num_angles(0)
    out = {}
    for kernel in (0, 1):
        sam.set_score_kernel(kernel)
        m = torch.full((nth, h, w), float("nan"), dtype=torch.float32, device="cuda")
        sam.score_map(model, 0, f, w, h, sam.FP32, m, 1, 1, 3, 0.0, 0, layout=sam.LAYOUT_PAIRS)
        torch.cuda.synchronize()
        out[kernel] = m.cpu().numpy()
    sam.set_score_kernel(0)
    assert sam.take_device_error() == 0
    assert np.abs(out[0] - out[1]).max() < TOL


def test_chunked_early_termination_exact_safe(big_case):
    tmpl, img, poses, model, om = big_case
    h, w = img.shape
    f = _pairs_field(img, 30, sam.FP32)
    x, y, th = poses[1]
    k = int(round(th / 0.5)) % 720
    win = (int(x) - 48, int(y) - 48, 96, 96, min(max(0, k - 3), 713), 7)
    full = _window(model, f, img, sam.FP32, win, early=0)
    for ms in (0.3, 0.6, 0.9):
        pr = _window(model, f, img, sam.FP32, win, early=1, min_score=ms)
        keep = full >= ms
        assert np.array_equal(pr[keep], full[keep])
        assert (pr[~keep] == full[~keep]).sum() + np.isneginf(pr[~keep]).sum() == (~keep).sum()
        assert np.isneginf(pr).any() or ms < 0.5


@pytest.mark.parametrize("prec", [sam.BF16, sam.FP16])
def test_chunked_16bit_with_fp32_rescoring(big_case, prec):
    tmpl, img, poses, model, om = big_case
    h, w = img.shape
    x, y, th = poses[0]
    k = int(round(th / 0.5)) % 720
    win = (int(x) - 64, int(y) - 40, 128, 80, min(max(0, k - 4), 711), 9)
    f32 = _window(model, _pairs_field(img, 30, sam.FP32), img, sam.FP32, win)
    f16 = _pairs_field(img, 30, prec)
    field32 = _pixel_field32(img, 30)
    ms = 0.5
    scratch = torch.empty(sam.score_window_scratch_bytes(1 << 20), dtype=torch.uint8, device="cuda")
    got = _window(model, f16, img, prec, win, early=1, min_score=ms, field32=field32, scratch=scratch)
    reach = f32 >= ms
    assert reach.any()
    assert np.abs(got[reach] - f32[reach]).max() < TOL
    # every pose left at a 16-bit value or -inf is below min_score in FP32
    assert (f32[~np.isfinite(got)] < ms).all()
    raw = _window(model, f16, img, prec, win, early=0)
    assert np.abs(raw - f32).max() < (6e-3 if prec == sam.BF16 else 8e-4)
    # a rescoring list too small for the window flags the overflow with NaN
    tiny = torch.empty(sam.score_window_scratch_bytes(4), dtype=torch.uint8, device="cuda")
    got2 = _window(model, f16, img, prec, win, early=0, min_score=0.0, field32=field32, scratch=tiny)
    assert np.isnan(got2).sum() == got2.size - 4


def test_detect_with_chunked_top_level(big_case):
    # one pyramid level: the exhaustive search runs at full resolution with
    # the chunked kernel; each detection's score is the oracle's at its pose
    tmpl, img, poses, model, om = big_case
    sub = np.ascontiguousarray(img)
    params = sam.default_detect_params(min_score=0.5, neighbourhood=3, top_k=16, max_detections=4)
    dets = sam.detect(model, _dev(sub), params)
    ofield = oracle.search_fields(sub, 1, 30)[0]
    assert len(dets) >= 1
    for d in dets:
        rot = oracle.rotate_points(om.points[0], d["k"], 0.5)
        ref = oracle.score_pose(ofield, rot, d["x"], d["y"], nbhd=3)
        assert abs(float(d["score"]) - ref) < TOL
    found = [any(abs(d["x"] - x) <= 2 and abs(d["y"] - y) <= 2 for d in dets) for x, y, _ in poses]
    assert any(found)


def test_angle_blocks_with_library_steps_merge_to_full_search(big_case):
    # the per-rank steps of an angle-sharded search (windowed scoring of a
    # block with its halo angles, candidate kernels), run here block by
    # block, merge to the candidates of the whole search
    from paper_2112_05576_gb300 import shard
    tmpl, img, poses, model, om = big_case
    x, y, _ = poses[0]
    sub = np.ascontiguousarray(img[int(y) - 200:int(y) + 200, int(x) - 200:int(x) + 200])
    h, w = sub.shape
    nth = model.num_angles(0)
    f = _pairs_field(sub, 30, sam.FP32)
    score_fn = shard.gpu_score_fn(model, 0, f, w, h, sam.FP32)
    cand_fn = shard.gpu_candidates_fn()
    K = 16
    full = score_fn(0, nth)
    ks, ys, xs, ss = cand_fn(full, 0.05, K)
    want = [(int(k), int(y), int(x), float(s)) for k, y, x, s in zip(ks, ys, xs, ss)]
    assert len(want) == K and abs(want[0][1] - 200) <= 1 and abs(want[0][2] - 200) <= 1
    for world in (2, 5):
        lists = [shard.block_candidates(*shard.angle_block(nth, world, r), nth, h, w, 0.05, K, score_fn, cand_fn)
                 for r in range(world)]
        assert shard.merge_candidates(lists, K, h, w) == want


def test_tiled_window_early_termination_exact_safe(small_case):
    # the tiled scorer over a pose window runs in one launch (bound pass,
    # then the surviving slices drained by the same CTA): every pose proved
    # below min_score is -inf and below it in the oracle, every other pose
    # matches the oracle, and no pose at or above min_score is pruned
    tmpl, img, model = small_case
    truth = synth.config1_scene()[2]
    om = oracle.create_model(tmpl, 30, 60, 1, 4.0)
    ofield = oracle.search_fields(img, 1, 30)[0]
    k0 = int(round(truth[0][2] / 4.0)) % 90 - 1
    ref = oracle.score_map_range(ofield, om.points[0], k0, 3, om.dtheta(0), nbhd=3, polarity=om.polarity)
    f = _pairs_field(img, 30, sam.FP32)
    h, w = img.shape
    sam.set_score_kernel(2, 2, 1, 3, 8)
    try:
        for win in ((0, 0, w, h, k0, 3), (37, 11, 201, 157, k0 + 1, 2)):
            x0, y0, gw, gh, wk0, nk = win
            sl = ref[wk0 - k0:wk0 - k0 + nk, y0:y0 + gh, x0:x0 + gw]
            for ms in (0.5, 0.7):
                got = _window(model, f, img, sam.FP32, win, early=1, min_score=ms)
                pruned = np.isneginf(got)
                assert pruned.any() and not pruned.all()
                assert np.all(sl[pruned] < ms)
                assert not np.any(pruned & (sl >= ms))
                assert np.max(np.abs(got[~pruned] - sl[~pruned])) < TOL
    finally:
        sam.set_score_kernel(0)

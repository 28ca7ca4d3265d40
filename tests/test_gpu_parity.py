"""GPU parity: every step of the CUDA path against the FP64 oracle.

Integers (pyramid, Sobel gradients, edge masks, candidate selection on the
same map) must be bit-exact; FP32 scores within 1e-5 absolute; BF16/FP16
stored fields within 2e-3; detections identical (pose and angle index) with
scores within 1e-5.
"""

import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

SCORE_TOL = 1e-5
# worst-case |M16 - M|: 2 sqrt(2) u per term (u = 2^-12 FP16, 2^-9 BF16) plus FP32 rounding
LOWP_TOL = {sam.FP16: 8e-4, sam.BF16: 6e-3}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()


# ---------------------------------------------------------------------------
# (b) pyramid
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("h,w", [(1024, 1280), (77, 301), (3, 2), (5, 33), (240, 320), (123, 4097)])
def test_pyramid_bit_exact(h, w):
    rng = np.random.default_rng(h * 7919 + w)
    img = rng.integers(0, 256, (h, w)).astype(np.uint8)
    src = _dev(img)
    dst = torch.zeros((h // 2, max(1, w // 2)), dtype=torch.uint8, device="cuda")
    sam.pyramid_down(src, dst)
    torch.cuda.synchronize()
    ref = oracle.pyramid_down(img)
    assert np.array_equal(dst.cpu().numpy()[:, : w // 2], ref)


def test_pyramid_strided_source():
    rng = np.random.default_rng(3)
    big = rng.integers(0, 256, (64, 200)).astype(np.uint8)
    src = _dev(big)[:, 10:171]       # width 161, stride 200
    dst = torch.zeros((32, 80), dtype=torch.uint8, device="cuda")
    sam.pyramid_down(src, dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), oracle.pyramid_down(big[:, 10:171]))


@pytest.mark.parametrize("h,w,levels", [(1024, 1280, 4), (77, 301, 4), (3, 2, 2), (5, 33, 3), (240, 320, 3),
                                          (123, 4097, 7), (1944, 2592, 5), (1, 1, 3), (130, 129, 8)])
def test_pyramid_levels_bit_exact(h, w, levels):
    # all levels in one launch equal levels - 1 oracle steps (floors of odd
    # sizes, block edges of the fused kernel, the per-level fallback at 8)
    rng = np.random.default_rng(h * 31 + w * 7 + levels)
    img = rng.integers(0, 256, (h, w)).astype(np.uint8)
    src = _dev(img)
    dsts = [torch.full((max(1, h >> l), max(1, w >> l) + 13), 77, dtype=torch.uint8, device="cuda")
            for l in range(1, levels)]
    sam.pyramid_levels(src, dsts)
    torch.cuda.synchronize()
    ref = img
    for l, d in enumerate(dsts, start=1):
        ref = oracle.pyramid_down(ref)
        got = d.cpu().numpy()
        assert np.array_equal(got[: h >> l, : w >> l], ref), l
        assert (got[:, w >> l:] == 77).all()   # nothing written past the level's width


# ---------------------------------------------------------------------------
# (a) gradient / threshold / normalise
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("h,w", [(1024, 1280), (77, 301), (3, 3), (16, 128), (17, 129), (240, 320), (61, 8)])
@pytest.mark.parametrize("low", [1, 30])
def test_gradient_bit_exact_and_field(h, w, low):
    rng = np.random.default_rng(h + 31 * w + low)
    img = rng.integers(0, 256, (h, w)).astype(np.uint8)
    src = _dev(img)
    field = torch.empty((h, w, 2), dtype=torch.float32, device="cuda")
    gx = torch.empty((h, w), dtype=torch.int16, device="cuda")
    gy = torch.empty((h, w), dtype=torch.int16, device="cuda")
    sam.gradient(src, low, sam.FP32, field, gx, gy)
    torch.cuda.synchronize()
    rgx, rgy = oracle.sobel(img)
    assert np.array_equal(gx.cpu().numpy(), rgx) and np.array_equal(gy.cpu().numpy(), rgy)
    mask = oracle.search_mask(rgx, rgy, low)
    rf = oracle.unit_field(rgx, rgy, mask)
    f = field.cpu().numpy()
    assert np.array_equal((np.abs(f).sum(-1) > 0), mask.astype(bool))
    assert np.max(np.abs(f - rf)) < 5e-7
    for prec, tol in ((sam.BF16, 2.0 ** -8), (sam.FP16, 2.0 ** -11)):
        hf = torch.empty((h, w, 2), dtype=torch.bfloat16 if prec == sam.BF16 else torch.float16, device="cuda")
        sam.gradient(src, low, prec, hf)
        torch.cuda.synchronize()
        g = hf.float().cpu().numpy()
        assert np.array_equal((np.abs(g).sum(-1) > 0), mask.astype(bool))
        assert np.max(np.abs(g - rf)) <= tol


# ---------------------------------------------------------------------------
# (c) exhaustive score map
# ---------------------------------------------------------------------------

def _field_dev(img, low, precision=sam.FP32):
    h, w = img.shape
    dt = {sam.FP32: torch.float32, sam.BF16: torch.bfloat16, sam.FP16: torch.float16}[precision]
    f = torch.empty((h, w, 2), dtype=dt, device="cuda")
    sam.gradient(_dev(img), low, precision, f)
    return f


def _gpu_map(model, level, img, precision=sam.FP32, step=(1, 1), nbhd=3, min_score=0.0, early=0):
    h, w = img.shape
    f = _field_dev(img, model.params.low, precision)
    nth = model.num_angles(level)
    gh, gw = (h + step[1] - 1) // step[1], (w + step[0] - 1) // step[0]
    out = torch.full((nth, gh, gw), float("nan"), dtype=torch.float32, device="cuda")
    sam.score_map(model, level, f, w, h, precision, out, step[0], step[1], nbhd, min_score, early)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _cfg1():
    tm, sc, truth = synth.config1_scene()
    return tm, sc, truth


@pytest.mark.parametrize("nbhd,polarity", [(3, 0), (1, 0), (3, 1)])
def test_score_map_config1_top_level(nbhd, polarity):
    tm, sc, _ = _cfg1()
    m = sam.Model(tm, 30, 60, 3, 1.0, polarity)
    om = oracle.create_model(tm, 30, 60, 3, 1.0, polarity)
    top = oracle.pyramid(sc, 3)[2]
    got = _gpu_map(m, 2, top, nbhd=nbhd)
    f = oracle.search_fields(sc, 3, 30)[2]
    ref = oracle.score_map(f, om.points[2], om.ntheta(2), om.dtheta(2), nbhd=nbhd, polarity=polarity)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < SCORE_TOL


def test_score_map_level0_small_and_step_grid():
    tm, sc, _ = synth.tiny_case(77, size=48, tsize=11)
    m = sam.Model(tm, 10, 20, 1, 15.0)
    om = oracle.create_model(tm, 10, 20, 1, 15.0)
    f = oracle.search_fields(sc, 1, 10)[0]
    for step in ((1, 1), (2, 3), (5, 1)):
        got = _gpu_map(m, 0, sc, step=step)
        ref = oracle.score_map(f, om.points[0], 24, 15.0, step_x=step[0], step_y=step[1])
        assert np.max(np.abs(got - ref)) < SCORE_TOL, step


def test_score_map_early_termination_is_exact_safe():
    tm, sc, _ = _cfg1()
    m = sam.Model(tm, 30, 60, 3, 1.0)
    om = oracle.create_model(tm, 30, 60, 3, 1.0)
    top = oracle.pyramid(sc, 3)[2]
    f = oracle.search_fields(sc, 3, 30)[2]
    ref = oracle.score_map(f, om.points[2], om.ntheta(2), om.dtheta(2))
    for ms in (0.5, 0.7, 0.9):
        got = _gpu_map(m, 2, top, min_score=ms, early=1)
        pruned = np.isneginf(got)
        assert pruned.sum() > 0
        assert np.all(ref[pruned] < ms), "a pruned pose reaches min_score"
        assert np.max(np.abs(got[~pruned] - ref[~pruned])) < SCORE_TOL


@pytest.mark.parametrize("precision", [sam.BF16, sam.FP16])
def test_score_map_low_precision_field(precision):
    tm, sc, _ = _cfg1()
    m = sam.Model(tm, 30, 60, 3, 1.0)
    om = oracle.create_model(tm, 30, 60, 3, 1.0)
    top = oracle.pyramid(sc, 3)[2]
    got = _gpu_map(m, 2, top, precision=precision)
    f = oracle.search_fields(sc, 3, 30)[2]
    ref = oracle.score_map(f, om.points[2], om.ntheta(2), om.dtheta(2))
    assert np.max(np.abs(got - ref)) < LOWP_TOL[precision]


# ---------------------------------------------------------------------------
# (d) candidates
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,K", [((1, 9, 13), 8), ((4, 17, 33), 64), ((45, 128, 160), 64), ((3, 1, 1), 4),
                                     ((2, 40, 3), 1000)])
def test_candidates_bit_exact_with_ties(shape, K):
    rng = np.random.default_rng(int(np.prod(shape)) + K)
    smap = (rng.integers(0, 9, shape) / 8.0).astype(np.float32)
    nth, gh, gw = shape
    d = _dev(smap)
    kyx = torch.zeros(3 * K, dtype=torch.int32, device="cuda")
    s = torch.zeros(K, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(sam.candidates_scratch_bytes(nth, gh, gw), dtype=torch.uint8, device="cuda")
    for _ in range(2):   # a second call must give the same answer (counters reset)
        sam.candidates(d, 0.5, K, kyx, s, cnt, scratch)
        torch.cuda.synchronize()
        n = int(cnt.item())
        ck, cy, cx, cs = oracle.candidates(smap.astype(np.float64), 0.5, K)
        assert n == len(ck)
        got = kyx.cpu().numpy()[: 3 * n].reshape(-1, 3)
        assert np.array_equal(got[:, 0], ck) and np.array_equal(got[:, 1], cy) and np.array_equal(got[:, 2], cx)
        assert np.array_equal(s.cpu().numpy()[:n], cs.astype(np.float32))


# ---------------------------------------------------------------------------
# full detection
# ---------------------------------------------------------------------------

def _compare_detections(got, ref, tol=SCORE_TOL):
    assert len(got) == len(ref), (got, ref)
    for g, r in zip(got, ref):
        assert (g["x"], g["y"], g["k"]) == (r[0], r[1], r[4]), (g, r)
        assert abs(g["score"] - r[3]) < tol, (g, r)


@pytest.mark.parametrize("nbhd", [3, 1])
def test_detect_config1_matches_oracle(nbhd):
    tm, sc, truth = _cfg1()
    m = sam.Model(tm, 30, 60, 3, 1.0)
    om = oracle.create_model(tm, 30, 60, 3, 1.0)
    ref = oracle.detect(om, sc, oracle.DetectParams(min_score=0.7, nbhd=nbhd))
    for early in (0, 1):
        p = sam.default_detect_params(min_score=0.7, neighbourhood=nbhd, early_termination=early)
        got_host = sam.detect(m, sc, p)
        got_dev = sam.detect(m, _dev(sc), p)
        _compare_detections(got_host, ref)
        _compare_detections(got_dev, ref)


def test_detect_config2_matches_oracle_and_truth():
    tm, sc, truth, _ = synth.config2_scene()
    m = sam.Model(tm, 30, 60, 4, 1.0)
    om = oracle.create_model(tm, 30, 60, 4, 1.0)
    ref = oracle.detect(om, sc, oracle.DetectParams(min_score=0.6, nbhd=3))
    got = sam.detect(m, _dev(sc), sam.default_detect_params(min_score=0.6))
    _compare_detections(got, ref)
    for gx, gy, gth in truth:
        near = [d for d in got if math.hypot(d["x"] - gx, d["y"] - gy) <= 2.0]
        if near:
            dth = abs((near[0]["theta_deg"] - gth + 180) % 360 - 180)
            assert dth <= 3.0


def test_detect_batch_equals_single():
    imgs = []
    tm, spec = None, None
    for i in range(3):
        t, sc, _, spec = synth.config2_scene(seed=3234 + i, W=640, H=480, spec=spec)
        tm = t if tm is None else tm
        imgs.append(sc)
    m = sam.Model(tm, 30, 60, 3, 1.0)
    p = sam.default_detect_params(min_score=0.5)
    batch = _dev(np.stack(imgs))
    got = sam.detect_batch(m, batch, p)
    for i, sc in enumerate(imgs):
        single = sam.detect(m, _dev(sc), p)
        assert got[i] == single
    # host input (the library copies the batch in): numpy, pinned torch, and
    # a strided host view, with graph mode on and off
    host = np.stack(imgs)
    wide = np.zeros((3, 480, 700), np.uint8)
    wide[:, :, :640] = host
    for graph in (1, 0):
        sam.set_graph_mode(graph)
        assert sam.detect_batch(m, host, p) == got
        assert sam.detect_batch(m, torch.from_numpy(host).pin_memory(), p) == got
        assert sam.detect_batch(m, torch.from_numpy(wide)[:, :, :640], p) == got
        assert sam.detect_batch(m, batch, p) == got
    sam.set_graph_mode(1)


def test_detect_edge_cases():
    tm, sc, _ = _cfg1()
    m = sam.Model(tm, 30, 60, 3, 1.0)
    flat = np.full((240, 320), 100, np.uint8)
    assert sam.detect(m, flat, sam.default_detect_params()) == []
    # image just large enough for the pyramid, far smaller than the template
    tiny = np.random.default_rng(0).integers(0, 256, (4, 4)).astype(np.uint8)
    om = oracle.create_model(tm, 30, 60, 3, 1.0)
    _compare_detections(sam.detect(m, tiny, sam.default_detect_params(min_score=0.1)),
                        oracle.detect(om, tiny, oracle.DetectParams(min_score=0.1)))
    # one candidate, one detection
    p = sam.default_detect_params(min_score=0.7, top_k=1, max_detections=1)
    ref = oracle.detect(om, sc, oracle.DetectParams(min_score=0.7, top_k=1, max_detections=1))
    _compare_detections(sam.detect(m, sc, p), ref)
    # nothing can reach 1.0 + a hair
    assert sam.detect(m, sc, sam.default_detect_params(min_score=1.0)) == \
        [] or all(d["score"] >= 1.0 for d in sam.detect(m, sc, sam.default_detect_params(min_score=1.0)))
    with pytest.raises(sam.SamError):
        sam.detect(m, sc, sam.default_detect_params(neighbourhood=5))

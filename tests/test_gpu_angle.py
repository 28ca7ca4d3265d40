"""GPU parity of the angle-only 16-bit field storage (SAM_ANGLE16).

The search field keeps only the direction of each edge gradient, as a 16-bit
code (edge bit + the angle rounded to 2 pi / 32768).  Against the FP64
oracle:

  * the codes are bit-exact (oracle.angle_codes on the same integer Sobel
    gradients), in both code layouts, on scenes, pyramid levels, noise and
    ragged sizes;
  * the scores of the code field (the tiled scorer stages the codes and
    expands them in shared memory) are within 1e-5 of the oracle's Eq. (1)
    on the field the codes stand for (oracle.angle_field), and within the
    storage bound 2 sin(pi / 65536) < 9.6e-5 (plus the same 1e-5) of the
    oracle's score of the exact unit field;
  * early termination stays exact-safe, in the one-CTA-per-unit form and in
    the persistent form;
  * calls the codes cannot serve are rejected.
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
STORAGE_BOUND = 2 * math.sin(math.pi / 65536)   # 9.59e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    yield
    sam.set_score_kernel(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _codes(img, low, layout=sam.LAYOUT_PAIRS):
    h, w = img.shape
    c = sam.angle_codes(_dev(img), low, layout=layout)
    torch.cuda.synchronize()
    out = c.cpu().numpy().view(np.uint16)
    assert out.shape == (h, sam.field_pitch(w, layout, sam.ANGLE16))
    if layout == sam.LAYOUT_PAIRS:
        assert not out[:, w:].any()     # padding codes are 0
    return out[:, :w]


def _oracle_codes(img, low):
    gx, gy = oracle.sobel(img)
    return oracle.angle_codes(gx, gy, low)


# ---------------------------------------------------------------------------
# the encoder (gradient kernel, SAM_ANGLE16)
# ---------------------------------------------------------------------------

def test_codes_bit_exact_on_scenes_and_levels():
    tm, sc, _, _ = synth.config2_scene()
    for lvl_img in oracle.pyramid(sc, 4):
        for layout in (sam.LAYOUT_PAIRS, sam.LAYOUT_PIXEL):
            assert np.array_equal(_codes(lvl_img, 30, layout), _oracle_codes(lvl_img, 30))
    tm1, sc1, _ = synth.config1_scene()
    for img in (tm1, sc1, tm):
        assert np.array_equal(_codes(img, 30), _oracle_codes(img, 30))


@pytest.mark.parametrize("h,w", [(1, 1), (3, 2), (7, 13), (61, 77), (128, 301), (257, 1030)])
def test_codes_bit_exact_on_noise_and_ragged_sizes(h, w):
    rng = np.random.default_rng(h * 1000 + w)
    img = rng.integers(0, 256, (h, w)).astype(np.uint8)
    for low in (1, 30):
        got = _codes(img, low)
        ref = _oracle_codes(img, low)
        assert np.array_equal(got, ref), (h, w, low)


def test_codes_cover_every_direction_of_a_disc():
    # a bright disc on a dark background: gradients of every direction,
    # including the axis codes 0, 8192, 16384 and 24576
    yy, xx = np.mgrid[0:400, 0:400].astype(np.float64)
    img = np.where((xx - 199.5) ** 2 + (yy - 199.5) ** 2 < 150.0 ** 2, 200, 40).astype(np.uint8)
    got = _codes(img, 10)
    assert np.array_equal(got, _oracle_codes(img, 10))
    a = got[got != 0] & 0x7FFF
    assert {0, 8192, 16384, 24576} <= set(np.unique(a).tolist())


# ---------------------------------------------------------------------------
# the scorer (staged codes, expanded in shared memory)
# ---------------------------------------------------------------------------

def _score(model, level, img, cfg=None, min_score=0.0, early=0, window=None, nbhd=3):
    h, w = img.shape
    if cfg is None:
        sam.set_score_kernel(0)
    else:
        sam.set_score_kernel(2, *cfg)
    codes = sam.angle_codes(_dev(img), model.params.low)
    nth = model.num_angles(level)
    if window is None:
        out = torch.full((nth, h, w), float("nan"), dtype=torch.float32, device="cuda")
        sam.score_map(model, level, codes, w, h, sam.ANGLE16, out, 1, 1, nbhd, min_score, early,
                      layout=sam.LAYOUT_PAIRS)
    else:
        x0, y0, gw, gh, k0, nk = window
        out = torch.full((nk, gh, gw), float("nan"), dtype=torch.float32, device="cuda")
        sam.score_window(model, level, codes, w, h, sam.ANGLE16, x0, y0, gw, gh, k0, nk, out, nbhd=nbhd,
                         min_score=min_score, early=early)
    torch.cuda.synchronize()
    assert sam.take_device_error() == 0
    return out.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def cfg2_top():
    tm, sc, _, _ = synth.config2_scene()
    m = sam.Model(tm, 30, 60, 4, 1.0)
    om = oracle.create_model(tm, 30, 60, 4, 1.0)
    top = oracle.pyramid(sc, 4)[3]
    codes = _oracle_codes(top, 30)
    ref_codes = oracle.score_map(oracle.angle_field(codes), om.points[3], om.ntheta(3), om.dtheta(3))
    ref_exact = oracle.score_map(oracle.search_fields(top, 1, 30)[0], om.points[3], om.ntheta(3), om.dtheta(3))
    return m, top, ref_codes, ref_exact


@pytest.mark.parametrize("cfg", [None, (1, 1, 3, 8), (2, 2, 1, 4), (1, 2, 45, 8), (1, 1, 3, 4, 10), (2, 1, 5, 8, 10)])
def test_angle_scores_match_oracle(cfg2_top, cfg):
    m, top, ref_codes, ref_exact = cfg2_top
    got = _score(m, 3, top, cfg)
    assert np.isfinite(got).all()
    assert np.max(np.abs(got - ref_codes)) < SCORE_TOL
    assert np.max(np.abs(got - ref_exact)) < STORAGE_BOUND + SCORE_TOL


@pytest.mark.parametrize("early_form", ["persistent", "per_unit"])
def test_angle_early_termination_exact_safe(cfg2_top, early_form):
    m, top, ref_codes, _ = cfg2_top
    h, w = top.shape
    for ms in (0.5, 0.6):
        if early_form == "persistent":    # sam_score_map: the persistent scorer with its task queue
            got = _score(m, 3, top, None, min_score=ms, early=1)
            ref = ref_codes
        else:                             # sam_score_window: one CTA per work unit
            win = (3, 5, w - 7, h - 9, 2, 40)
            got = _score(m, 3, top, None, min_score=ms, early=1, window=win)
            ref = ref_codes[2:42, 5:5 + h - 9, 3:3 + w - 7]
        pruned = np.isneginf(got)
        assert pruned.any() and not pruned.all()
        assert np.all(ref[pruned] < ms)
        assert np.max(np.abs(got[~pruned] - ref[~pruned])) < SCORE_TOL


@pytest.mark.parametrize("nbhd,polarity", [(1, 0), (3, 1), (1, 1)])
def test_angle_scores_neighbourhood_and_polarity(nbhd, polarity):
    tm, sc, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, 3, 1.0, polarity=polarity)
    om = oracle.create_model(tm, 30, 60, 3, 1.0, polarity=polarity)
    img = oracle.pyramid(sc, 3)[2]
    got = _score(m, 2, img, nbhd=nbhd)
    ref = oracle.score_map(oracle.angle_field(_oracle_codes(img, 30)), om.points[2], om.ntheta(2), om.dtheta(2),
                           nbhd=nbhd, polarity=polarity)
    assert np.max(np.abs(got - ref)) < SCORE_TOL


@pytest.mark.parametrize("h,w", [(61, 77), (7, 5), (1, 1), (33, 130)])
def test_angle_scores_ragged_and_tiny(h, w):
    tm, sc, _ = synth.tiny_case(h * 100 + w, size=max(h, w, 24), tsize=11)
    img = np.ascontiguousarray(sc[:h, :w])
    m = sam.Model(tm, 10, 20, 1, 15.0)
    om = oracle.create_model(tm, 10, 20, 1, 15.0)
    got = _score(m, 0, img, (1, 1, 5, 4))
    ref = oracle.score_map(oracle.angle_field(_oracle_codes(img, 10)), om.points[0], 24, 15.0)
    assert np.max(np.abs(got - ref)) < SCORE_TOL, (h, w)


def test_angle_rejects_what_it_cannot_serve(cfg2_top):
    m, top, _, _ = cfg2_top
    h, w = top.shape
    codes = sam.angle_codes(_dev(top), 30)
    out = torch.empty((m.num_angles(3), h, w), dtype=torch.float32, device="cuda")
    sam.set_score_kernel(0)
    with pytest.raises(sam.SamError):   # step 2: no generic scorer for codes
        sam.score_map(m, 3, codes, w, h, sam.ANGLE16, out, 2, 2, 3, 0.0, 0, layout=sam.LAYOUT_PAIRS)
    with pytest.raises(sam.SamError):   # pixel layout: not the TMA-read layout
        sam.score_map(m, 3, codes, w, h, sam.ANGLE16, out, 1, 1, 3, 0.0, 0, layout=sam.LAYOUT_PIXEL)
    with pytest.raises(sam.SamError):   # detection does not take codes
        sam.detect(m, torch.from_numpy(np.zeros((64, 64), np.uint8)).cuda(),
                   sam.default_detect_params(precision=sam.ANGLE16))

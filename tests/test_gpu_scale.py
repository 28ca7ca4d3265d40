"""GPU parity of the scaled-pose search (Eq. (2) with A = s R(theta)).

A scaled model carries one table per (scale, angle); its score maps have
num_scales x num_angles planes, its candidates are local maxima over
(scale, angle, y, x) and its descent searches the scale +- 1 as well.
Against the FP64 oracle (oracle.score_map_scaled, candidates_scaled,
detect_scaled):

  * the score map of every scorer (tiled, generic, with early termination,
    a pose window) is within 1e-5 of Eq. (1) over the scaled projections;
  * candidates are bit-exact on tied maps;
  * full detections of scenes with instances at several scales are the
    oracle's (x, y, angle, scale identical, scores within 1e-5), and find
    the rendered instances at their scale;
  * a template enlarged 2x by pixel replication is found at scale 2 with
    score 1;
  * entry points that take rigid poses only reject scaled models.
"""

import numpy as np
import pytest

import oracle
import synth
import _oracle_pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

SCORE_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    sam.set_score_kernel(0)
    yield
    sam.set_score_kernel(0)
    sam.set_graph_mode(True)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(got, ref, what=""):
    assert len(got) == len(ref), (what, got, ref)
    for g, r in zip(got, ref):
        assert (g["x"], g["y"], g["k"], g["j"]) == (r[0], r[1], r[4], r[5]), (what, g, r)
        assert abs(g["score"] - r[3]) < SCORE_TOL, (what, g, r)


# ---------------------------------------------------------------------------
# score maps
# ---------------------------------------------------------------------------

SCALES = (0.8, 0.2, 3)


@pytest.fixture(scope="module")
def map_case():
    tm, sc, _ = synth.config1_scene()
    img = oracle.pyramid(sc, 2)[1]                    # 160 x 120
    m = sam.Model(tm, 30, 60, 1, 12.0, scales=SCALES)
    om = oracle.create_model(tm, 30, 60, 1, 12.0)
    field = oracle.search_fields(img, 1, 30)[0]
    ref = oracle.score_map_scaled(field, om.points[0], oracle.scale_grid(*SCALES), om.ntheta(0), om.dtheta(0))
    return m, img, ref


def _scaled_map(m, img, kernel=0, cfg=(1, 1, 3, 8), min_score=0.0, early=0):
    h, w = img.shape
    sam.set_score_kernel(kernel, *cfg) if kernel else sam.set_score_kernel(0)
    wp = sam.field_pitch(w, sam.LAYOUT_PAIRS)
    f = torch.zeros((h, wp, 2), dtype=torch.float32, device="cuda")
    sam.gradient(_dev(img), 30, sam.FP32, f, layout=sam.LAYOUT_PAIRS)
    planes = m.num_scales() * m.num_angles(0)
    out = torch.full((planes, h, w), float("nan"), dtype=torch.float32, device="cuda")
    sam.score_map(m, 0, f, w, h, sam.FP32, out, 1, 1, 3, min_score, early, layout=sam.LAYOUT_PAIRS)
    torch.cuda.synchronize()
    assert sam.take_device_error() == 0
    return out.cpu().numpy().reshape(m.num_scales(), m.num_angles(0), h, w).astype(np.float64)


@pytest.mark.parametrize("kernel,cfg", [(0, None), (1, (1, 1, 3, 8)), (2, (1, 1, 3, 8)), (2, (2, 1, 5, 8, 10)),
                                        (2, (2, 2, 0, 4))])
def test_scaled_score_map_matches_oracle(map_case, kernel, cfg):
    m, img, ref = map_case
    got = _scaled_map(m, img, kernel, cfg or (1, 1, 3, 8))
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < SCORE_TOL


def test_scaled_score_map_early_termination_exact_safe(map_case):
    m, img, ref = map_case
    for ms in (0.5, 0.7):
        got = _scaled_map(m, img, 0, min_score=ms, early=1)
        pruned = np.isneginf(got)
        assert pruned.any() and not pruned.all()
        assert np.all(ref[pruned] < ms)
        assert np.max(np.abs(got[~pruned] - ref[~pruned])) < SCORE_TOL


# ---------------------------------------------------------------------------
# candidates
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,K", [((3, 45, 40, 50), 64), ((5, 8, 16, 20), 200), ((2, 1, 9, 7), 30),
                                     ((1, 30, 20, 20), 50)])
def test_candidates_scaled_bit_exact(shape, K):
    rng = np.random.default_rng(int(np.prod(shape)) + K)
    smap = (rng.integers(0, 9, shape) / 8.0).astype(np.float32)
    ns, na, gh, gw = shape
    d = _dev(smap)
    kyx = torch.zeros(3 * K, dtype=torch.int32, device="cuda")
    s = torch.zeros(K, dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = torch.empty(sam.candidates_scaled_scratch_bytes(ns, na, gh, gw), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        sam.candidates_scaled(d, 0.5, K, kyx, s, cnt, scratch)
        torch.cuda.synchronize()
        n = int(cnt.item())
        cj, ck, cy, cx, cs = oracle.candidates_scaled(smap.astype(np.float64), 0.5, K)
        assert n == len(cj)
        got = kyx.cpu().numpy()[: 3 * n].reshape(-1, 3)
        assert np.array_equal(got[:, 0], cj * na + ck)
        assert np.array_equal(got[:, 1], cy) and np.array_equal(got[:, 2], cx)
        assert np.array_equal(s.cpu().numpy()[:n], cs.astype(np.float32))


# ---------------------------------------------------------------------------
# detection
# ---------------------------------------------------------------------------

DET_SCALES = (0.85, 0.15, 3)      # 0.85, 1.0, 1.15


@pytest.fixture(scope="module")
def det_case():
    grid = oracle.scale_grid(*DET_SCALES)
    scenes, tm, spec = [], None, None
    for i in range(3):
        t, sc, gts, spec = synth.config2_scene(seed=7700 + i, W=640, H=512, side=96, spec=spec, n_inst=2,
                                               scales=grid)
        tm = t if tm is None else tm
        scenes.append((sc, gts))
    ref = _oracle_pool.detect_scaled_many([(tm, sc, (30, 60, 3, 1.0), grid,
                                            dict(min_score=0.6, nbhd=3, top_k=64, max_detections=16))
                                           for sc, _ in scenes])
    m = sam.Model(tm, 30, 60, 3, 1.0, scales=DET_SCALES)
    return m, scenes, ref, grid


def test_scaled_detection_matches_oracle(det_case):
    m, scenes, ref, grid = det_case
    p = sam.default_detect_params(min_score=0.6)
    assert sum(len(r) for r in ref) >= 3
    for graph in (True, False):
        sam.set_graph_mode(graph)
        for i, (sc, _) in enumerate(scenes):
            _same(sam.detect(m, _dev(sc), p), ref[i], (graph, i))
    sam.set_graph_mode(True)
    batch = sam.detect_batch(m, _dev(np.stack([sc for sc, _ in scenes])), p)
    for i in range(len(scenes)):
        _same(batch[i], ref[i], ("batch", i))


def test_scaled_detection_finds_instances_at_their_scale(det_case):
    # recovery of the rendered instances (not parity: the detections above
    # are the oracle's): found within 2 px, at their scale, and within the
    # coarse-to-fine window's angle reach
    m, scenes, ref, grid = det_case
    p = sam.default_detect_params(min_score=0.6)
    hits = right_scale = right_angle = 0
    for sc, gts in scenes:
        dets = sam.detect(m, _dev(sc), p)
        for gx, gy, gth, gs in gts:
            near = [d for d in dets if (d["x"] - gx) ** 2 + (d["y"] - gy) ** 2 <= 4]
            if near:
                hits += 1
                d = near[0]
                right_scale += int(m.scale(d["j"]) == pytest.approx(gs))
                right_angle += int(abs(((d["theta_deg"] - gth) + 180) % 360 - 180) <= 3.0)
    assert hits >= 4
    assert right_scale >= 0.8 * hits and right_angle >= 0.8 * hits


@pytest.mark.parametrize("levels", [1, 2])
def test_enlarged_template_found_at_scale_two(levels):
    tm = np.full((24, 24), 60, np.uint8)
    tm[6:18, 6:18] = 200
    tm[9:12, 9:15] = 60
    scene = np.full((80, 80), 60, np.uint8)
    scene[16:64, 16:64] = np.kron(tm, np.ones((2, 2), np.uint8))
    step = 90.0 if levels == 1 else 45.0
    scales = (1.0, 0.5, 4) if levels == 1 else (1.0, 0.5, 3)
    m = sam.Model(tm, 30, 60, levels, step, scales=scales)
    om = oracle.create_model(tm, 30, 60, levels, step)
    ref = oracle.detect_scaled(om, scene, oracle.DetectParams(min_score=0.5), oracle.scale_grid(*scales))
    got = sam.detect(m, _dev(scene), sam.default_detect_params(min_score=0.5))
    _same(got, ref)
    assert got[0]["j"] == 2 and abs(got[0]["score"] - 1.0) < SCORE_TOL
    assert got[0]["x"] in (40, 41) and got[0]["y"] in (40, 41)


def test_rigid_only_entry_points_reject_scaled_models():
    tm, sc, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, 3, 1.0, scales=(0.9, 0.1, 3))
    field = sam.unit_field(_dev(sc), 30)
    with pytest.raises(sam.SamError):
        sam.MultiPlan([m], [(320, 240)], [(0, 0)])
    with pytest.raises(sam.SamError):
        sam.subpixel_poses(m, [field], torch.tensor([[0, 100, 100]], dtype=torch.int32, device="cuda"))
    with pytest.raises(sam.SamError):
        sam.score_bilinear(m, [field], torch.tensor([[100.0, 100.0, 0.0]], device="cuda"))

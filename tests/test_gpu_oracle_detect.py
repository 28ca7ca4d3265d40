"""Detections of the batched paths against the FP64 oracle.

Sec. II returns the maximum score and its pose; these tests compare, pose by
pose, what the library's batched entry points return with what the oracle's
plain detection (oracle.detect: exhaustive top level, 27-pose refinement per
level, NMS) returns for the same scene:

  * the step the benchmark times: sam_detect_batch on a batch of sixteen
    1280x1024 config-2 scenes with early termination and the autotuned batch
    tiling, in FP32 and with BF16 / FP16 stored fields after the FP32
    rescoring of the top level;
  * an uneven batched plan (images of six sizes, templates with 3 and 4
    levels, one graph, the persistent pairs scorer): every pair's detections,
    and every pair's top-level score map element by element (finite entries
    within 1e-5 of Eq. (1), pruned entries below min_score in the oracle).

Bar: identical (x, y, angle index) and scores within 1e-5; the order may
differ only between detections whose scores are within 1e-5 of each other.
"""

import numpy as np
import pytest

import synth
import _oracle_pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

SCORE_TOL = 1e-5
MIN_SCORE = 0.6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    sam.set_score_kernel(0)
    yield
    sam.set_score_kernel(0)


def assert_same_detections(got, ref, tol=SCORE_TOL, what=""):
    """got: the binding's dicts; ref: oracle.detect tuples (x, y, theta, score, k)."""
    assert len(got) == len(ref), (what, got, ref)
    for i, (g, r) in enumerate(zip(got, ref)):
        if (g["x"], g["y"], g["k"]) == (r[0], r[1], r[4]):
            assert abs(g["score"] - r[3]) < tol, (what, i, g, r)
            continue
        # a swap is allowed only inside a group of scores tied within tol
        tied = [j for j, rr in enumerate(ref) if abs(rr[3] - r[3]) < tol]
        assert any((g["x"], g["y"], g["k"]) == (ref[j][0], ref[j][1], ref[j][4]) for j in tied), (what, i, g, r)
        assert abs(g["score"] - r[3]) < tol, (what, i, g, r)


# ---------------------------------------------------------------------------
# the benchmark's step: a batch of config-2 scenes, autotuned tiling
# ---------------------------------------------------------------------------

BATCH = 16


@pytest.fixture(scope="module")
def bench_batch():
    import bench
    tm, imgs, truth, _ = bench._scenes(BATCH, 3000)     # the benchmark's first batch
    jobs = [(tm, im, (bench.LOW, bench.HIGH, bench.LEVELS, bench.STEP),
             dict(min_score=bench.MIN_SCORE, nbhd=3, top_k=64, max_detections=16)) for im in imgs]
    ref = _oracle_pool.detect_many(jobs)
    model = sam.Model(tm, bench.LOW, bench.HIGH, bench.LEVELS, bench.STEP)
    dev = torch.from_numpy(np.stack(imgs)).cuda()
    return model, dev, ref, truth


@pytest.mark.parametrize("prec", [sam.FP32, sam.BF16, sam.FP16])
def test_bench_step_matches_oracle(bench_batch, prec):
    model, dev, ref, _ = bench_batch
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                       precision=prec, early_termination=1)
    tuned = sam.autotune(model, dev, params)
    assert tuned, "the autotuner timed no tiling"
    assert sum(len(r) for r in ref) >= BATCH
    for rep in range(2):   # the first call captures the pipeline graph, the second replays it
        got = sam.detect_batch(model, dev, params)
        for i, (g, r) in enumerate(zip(got, ref)):
            assert_same_detections(g, r, what=(prec, rep, i))


def test_bench_step_without_early_termination_matches_oracle(bench_batch):
    model, dev, ref, _ = bench_batch
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                       precision=sam.FP32, early_termination=0)
    got = sam.detect_batch(model, dev[:4], params)
    for i, (g, r) in enumerate(zip(got, ref[:4])):
        assert_same_detections(g, r, what=i)


# ---------------------------------------------------------------------------
# the uneven batched plan (one graph, persistent pairs scorer)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def plan_batch():
    rng = np.random.default_rng(4321)
    sides, levels = (48, 96, 200), (3, 3, 4)
    specs = [synth.random_part(rng, s, kind="part", margin=4.0) for s in sides]
    tmpls = [synth.render_template(s) for s in specs]
    models = [sam.Model(t, 30, 60, L, 1.0) for t, L in zip(tmpls, levels)]
    sizes = [(320, 240), (640, 480), (401, 301), (1280, 1024), (333, 257), (512, 512)]
    images, pairs = [], []
    for i, (w, h) in enumerate(sizes):
        which = [j for j in range(3) if specs[j].width * 1.6 < min(w, h)]
        spec = specs[which[-1]]
        _, img, _, _ = synth.config2_scene(seed=700 + i, W=w, H=h, side=spec.width, spec=spec,
                                           n_inst=int(rng.integers(1, 3)))
        images.append(img)
        for j in which[-2:]:
            pairs.append((i, j))
    margs = [(30, 60, L, 1.0) for L in levels]
    det_jobs = [(tmpls[j], images[i], margs[j], dict(min_score=MIN_SCORE, nbhd=3, top_k=64, max_detections=16))
                for i, j in pairs]
    map_jobs = [(tmpls[j], images[i], margs[j], 3) for i, j in pairs]
    ref = _oracle_pool.detect_many(det_jobs)
    maps = _oracle_pool.top_maps(map_jobs)
    return models, sizes, images, pairs, ref, maps


@pytest.mark.parametrize("prec", [sam.FP32, sam.FP16, sam.BF16])
def test_plan_matches_oracle(plan_batch, prec):
    models, sizes, images, pairs, ref, maps = plan_batch
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                       precision=prec, early_termination=1)
    plan = sam.MultiPlan(models, sizes, pairs, params)
    for i, img in enumerate(images):
        plan.set_image(i, torch.from_numpy(img).cuda())
    plan.autotune()
    assert sum(len(r) for r in ref) > 0
    for rep in range(2):
        got = plan.run()
        for p, (g, r) in enumerate(zip(got, ref)):
            assert_same_detections(g, r, what=(prec, rep, p, pairs[p]))
    # every pair's top-level map as the last run left it (a pair whose
    # template is absent from its image may have every pose pruned); a
    # 16-bit field's map holds its own scores, within the storage bound of
    # the FP32 ones (candidate extraction rescored the poses it decided on)
    tol = SCORE_TOL + {sam.FP32: 0.0, sam.FP16: 8e-4, sam.BF16: 6e-3}[prec]
    n_live = 0
    for p, om in enumerate(maps):
        gm, lvl = plan.pair_map(p)
        gm = gm.cpu().numpy().astype(np.float64)
        assert gm.shape == om.shape and lvl == models[pairs[p][1]].levels - 1
        pruned = np.isneginf(gm)
        assert np.all(om[pruned] < MIN_SCORE), (prec, p)
        live = ~pruned
        n_live += int(live.sum())
        if live.any():
            assert np.max(np.abs(gm[live] - om[live])) < tol, (prec, p)
    assert n_live > 0
    plan.close()


def test_plan_map_rejects_bad_pair(plan_batch):
    models, sizes, images, pairs, _, _ = plan_batch
    plan = sam.MultiPlan(models, sizes, pairs, sam.default_detect_params(min_score=MIN_SCORE))
    with pytest.raises(sam.SamError):
        plan.pair_map(len(pairs))
    with pytest.raises(sam.SamError):
        plan.pair_map(-1)
    plan.close()

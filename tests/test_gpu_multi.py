"""GPU parity of batched uneven detection (one graph, persistent scorer).

Every (image, model) pair of an uneven batch -- images of six sizes
including odd ones, models with 3 and 4 pyramid levels -- must give exactly
the detections of the single-image path for that pair (same poses, same
FP32 scores), on repeated graph replays, after autotuning the plan's tiling,
and with an FP16-stored field.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    sam.set_score_kernel(0)


def _key(dets):
    return [(d["x"], d["y"], d["k"], round(float(d["score"]), 6)) for d in dets]


@pytest.fixture(scope="module")
def batch():
    rng = np.random.default_rng(99)
    specs = [synth.random_part(rng, s, kind="part", margin=4.0) for s in (48, 96, 200)]
    tmpls = [synth.render_template(s) for s in specs]
    levels = [3, 3, 4]
    models = [sam.Model(t, 30, 60, L, 1.0) for t, L in zip(tmpls, levels)]
    sizes = [(320, 240), (640, 480), (401, 301), (1280, 1024), (333, 257), (512, 512)]
    images, pairs = [], []
    for i, (w, h) in enumerate(sizes):
        which = [j for j in range(3) if specs[j].width * 1.6 < min(w, h)]
        spec = specs[which[-1]]
        _, img, _, _ = synth.config2_scene(seed=500 + i, W=w, H=h, side=spec.width, spec=spec,
                                           n_inst=int(rng.integers(1, 3)))
        images.append(img)
        for j in which[-2:]:
            pairs.append((i, j))
    return models, sizes, images, pairs


def _single(models, images, pairs, params):
    return [sam.detect(models[m], torch.from_numpy(images[i]).cuda(), params) for i, m in pairs]


@pytest.mark.parametrize("prec", [sam.FP32, sam.FP16])
def test_plan_matches_single_image_path(batch, prec):
    models, sizes, images, pairs = batch
    params = sam.default_detect_params(min_score=0.6, precision=prec)
    plan = sam.MultiPlan(models, sizes, pairs, params)
    for i, img in enumerate(images):
        plan.set_image(i, torch.from_numpy(img).cuda())
    ref = _single(models, images, pairs, params)
    assert sum(len(r) for r in ref) > 0
    first = plan.run()
    assert [_key(d) for d in first] == [_key(d) for d in ref]
    again = plan.run()    # graph replay
    assert [_key(d) for d in again] == [_key(d) for d in ref]
    st = plan.stats()
    assert st["graph_kernels"] >= 8 and st["pose_points"] > 0
    plan.close()


def test_plan_autotune_and_tilings(batch):
    models, sizes, images, pairs = batch
    params = sam.default_detect_params(min_score=0.6)
    plan = sam.MultiPlan(models, sizes, pairs, params)
    for i, img in enumerate(images):
        plan.set_image(i, img)
    ref = [_key(d) for d in plan.run()]
    res = plan.autotune()
    assert len(res) >= 8 and all(ms > 0 for _, ms in res)
    assert [_key(d) for d in plan.run()] == ref
    for t in [(2, 2, 1, 4), (1, 1, 15, 8), (2, 1, 5, 8), (1, 1, 3, 8, 10), (2, 2, 5, 4, 10)]:
        plan.set_tiling(*t)
        assert [_key(d) for d in plan.run()] == ref
    plan.close()


def test_plan_rejects_bad_arguments(batch):
    models, sizes, images, pairs = batch
    with pytest.raises(sam.SamError):
        sam.MultiPlan(models, sizes, [(0, 7)])
    with pytest.raises(sam.SamError):
        sam.MultiPlan(models, sizes, pairs, sam.default_detect_params(step_x=2))
    with pytest.raises(sam.SamError):
        sam.MultiPlan(models, [(3, 3)], [(0, 2)])   # too small for 4 levels

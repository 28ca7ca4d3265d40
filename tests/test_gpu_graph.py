"""Graph mode: sam_detect / sam_detect_batch replay the whole pipeline as a
captured CUDA graph.  Results must be identical to the direct path's (same
poses, same FP32 scores) for single images from host and device memory and
for batches, across re-captures caused by a new shape, new parameters or a
new scorer tiling, and a replay must launch the same kernels as one direct
call.
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
    yield
    sam.set_graph_mode(True)
    sam.set_score_kernel(0)


def _key(dets):
    return [(d["x"], d["y"], d["k"], float(d["score"])) for d in dets]


@pytest.fixture(scope="module")
def scenes():
    imgs, tm, spec = [], None, None
    for i in range(4):
        t, sc, _, spec = synth.config2_scene(seed=8100 + i, spec=spec, W=640, H=512)
        tm = t if tm is None else tm
        imgs.append(sc)
    return tm, imgs


def _both(fn):
    sam.set_graph_mode(False)
    direct = fn()
    sam.set_graph_mode(True)
    first = fn()    # captures
    again = fn()    # replays
    return direct, first, again


def test_graph_equals_direct_single_and_batch(scenes):
    tm, imgs = scenes
    m = sam.Model(tm, 30, 60, 3, 1.0)
    p = sam.default_detect_params(min_score=0.6)
    dev = [torch.from_numpy(im).cuda() for im in imgs]
    batch = torch.stack(dev)
    for fn in (lambda: [sam.detect(m, dev[0], p)], lambda: [sam.detect(m, imgs[1], p)],
               lambda: sam.detect_batch(m, batch, p), lambda: sam.detect_batch(m, batch[1:3], p)):
        d, f, a = _both(fn)
        assert sum(len(x) for x in d) > 0
        assert [_key(x) for x in f] == [_key(x) for x in d]
        assert [_key(x) for x in a] == [_key(x) for x in d]


def test_graph_recaptures_on_changes(scenes):
    tm, imgs = scenes
    m = sam.Model(tm, 30, 60, 3, 1.0)
    batch = torch.stack([torch.from_numpy(im).cuda() for im in imgs])
    p1 = sam.default_detect_params(min_score=0.6)
    p2 = sam.default_detect_params(min_score=0.7, precision=sam.FP16)
    sam.set_graph_mode(False)
    ref1 = sam.detect_batch(m, batch, p1)
    ref2 = sam.detect_batch(m, batch, p2)
    sam.set_graph_mode(True)
    for _ in range(2):
        assert [_key(x) for x in sam.detect_batch(m, batch, p1)] == [_key(x) for x in ref1]
        assert [_key(x) for x in sam.detect_batch(m, batch, p2)] == [_key(x) for x in ref2]
    # a different scorer tiling invalidates the captured pipeline
    for cfg in [(1, 1, 3, 4, 10), (2, 2, 0, 4), (2, 1, 9, 8)]:
        sam.set_score_kernel(2, *cfg)
        sam.set_graph_mode(False)
        want = [_key(x) for x in sam.detect_batch(m, batch, p1)]
        sam.set_graph_mode(True)
        assert [_key(x) for x in sam.detect_batch(m, batch, p1)] == want
    sam.set_score_kernel(0)


def test_replay_launches_the_pipeline_kernels(scenes):
    tm, imgs = scenes
    m = sam.Model(tm, 30, 60, 3, 1.0)
    batch = torch.stack([torch.from_numpy(im).cuda() for im in imgs])
    p = sam.default_detect_params(min_score=0.6)
    sam.set_graph_mode(False)
    sam.detect_batch(m, batch, p)
    n0 = sam.kernel_launches()
    sam.detect_batch(m, batch, p)
    direct = sam.kernel_launches() - n0
    sam.set_graph_mode(True)
    sam.detect_batch(m, batch, p)   # capture
    n0 = sam.kernel_launches()
    sam.detect_batch(m, batch, p)
    assert sam.kernel_launches() - n0 == direct

"""GPU parity of the 16-bit stored forms (FP16 / BF16 w_hat, FP32 accumulation).

The stored unit field is rounded to 16 bits and the point direction to the
same type; the products are exact (mixed-precision FMA) and maxima and sums
stay FP32, so: the tiled and generic kernels agree to FP32 summation error
on the same 16-bit field, both stay within the worst-case storage bound of
the FP64 oracle (8e-4 FP16, 6e-3 BF16), early termination stays exact-safe
with the widened margin, and full detections (refined and rescored on FP32
fields) equal the FP32 path's.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

# worst-case |M16 - M| against exact arithmetic: 16-bit field and direction
# components rounded (2 sqrt(2) u per term, u = 2^-12 FP16, 2^-9 BF16) plus
# FP32 accumulation
LOWP = {sam.FP16: 8e-4, sam.BF16: 6e-3}
PRECS = [(sam.FP16, torch.float16), (sam.BF16, torch.bfloat16)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()
    yield
    sam.set_score_kernel(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _map(model, level, img, prec, dt, kernel, cfg=(1, 1, 3, 8), min_score=0.0, early=0):
    h, w = img.shape
    sam.set_score_kernel(kernel, *cfg)
    wp = sam.field_pitch(w, sam.LAYOUT_PAIRS)
    f = torch.zeros((h, wp, 2), dtype=dt, device="cuda")
    sam.gradient(_dev(img), model.params.low, prec, f, layout=sam.LAYOUT_PAIRS)
    out = torch.full((model.num_angles(level), h, w), float("nan"), dtype=torch.float32, device="cuda")
    sam.score_map(model, level, f, w, h, prec, out, 1, 1, 3, min_score, early, layout=sam.LAYOUT_PAIRS)
    torch.cuda.synchronize()
    assert sam.take_device_error() == 0
    return out.cpu().numpy()


@pytest.fixture(scope="module")
def cfg2():
    tm, sc, truth, _ = synth.config2_scene()
    m = sam.Model(tm, 30, 60, 4, 1.0)
    om = oracle.create_model(tm, 30, 60, 4, 1.0)
    top = oracle.pyramid(sc, 4)[3]
    f = oracle.search_fields(top, 1, 30)[0]
    ref = oracle.score_map(f, om.points[3], om.ntheta(3), om.dtheta(3))
    return tm, sc, m, top, ref


@pytest.mark.parametrize("prec,dt", PRECS)
@pytest.mark.parametrize("cfg", [(1, 1, 3, 8), (2, 2, 1, 4), (1, 2, 45, 8), (1, 1, 3, 4, 10), (2, 1, 5, 8, 10), (2, 2, 0, 4)])
def test_tiled_lowp_matches_generic_and_oracle(cfg2, prec, dt, cfg):
    _, _, m, top, ref = cfg2
    tiled = _map(m, 3, top, prec, dt, 2, cfg)
    generic = _map(m, 3, top, prec, dt, 1)
    assert np.max(np.abs(tiled - generic)) < 1e-5
    assert np.max(np.abs(tiled - ref)) < LOWP[prec]


@pytest.mark.parametrize("prec,dt", PRECS)
def test_tiled_lowp_ragged_and_tiny(prec, dt):
    for h, w in [(61, 77), (7, 5), (1, 1), (33, 130)]:
        tm, sc, _ = synth.tiny_case(h * 100 + w, size=max(h, w, 24), tsize=11)
        img = np.ascontiguousarray(sc[:h, :w])
        m = sam.Model(tm, 10, 20, 1, 15.0)
        om = oracle.create_model(tm, 10, 20, 1, 15.0)
        got = _map(m, 0, img, prec, dt, 2, (1, 1, 5, 4))
        gen = _map(m, 0, img, prec, dt, 1)
        f = oracle.search_fields(img, 1, 10)[0]
        ref = oracle.score_map(f, om.points[0], 24, 15.0)
        assert np.max(np.abs(got - gen)) < 1e-5, (h, w)
        assert np.max(np.abs(got - ref)) < LOWP[prec], (h, w)


@pytest.mark.parametrize("prec,dt", PRECS)
def test_tiled_lowp_early_termination_exact_safe(cfg2, prec, dt):
    _, _, m, top, ref = cfg2
    for ms in (0.5, 0.6):
        got = _map(m, 3, top, prec, dt, 2, min_score=ms, early=1)
        pruned = np.isneginf(got)
        assert pruned.any()
        assert np.all(ref[pruned] < ms)
        assert np.max(np.abs(got[~pruned] - ref[~pruned])) < LOWP[prec]


@pytest.mark.parametrize("prec", [sam.FP16, sam.BF16])
def test_lowp_detections_equal_fp32(prec):
    imgs, tm, spec = [], None, None
    for i in range(6):
        t, sc, _, spec = synth.config2_scene(seed=8200 + i, spec=spec)
        tm = t if tm is None else tm
        imgs.append(sc)
    m = sam.Model(tm, 30, 60, 4, 1.0)
    batch = _dev(np.stack(imgs))
    sam.set_score_kernel(0)
    ref = sam.detect_batch(m, batch, sam.default_detect_params(min_score=0.6))
    got = sam.detect_batch(m, batch, sam.default_detect_params(min_score=0.6, precision=prec))
    for a, b in zip(got, ref):
        assert [(d["x"], d["y"], d["k"]) for d in a] == [(d["x"], d["y"], d["k"]) for d in b]
        assert all(abs(x["score"] - y["score"]) < 1e-6 for x, y in zip(a, b))

"""GPU parity of the differentiable continuous-pose score, its adjoint and
the one-launch Gauss-Newton pose refinement, against the FP64 oracle.

Workload shaped like pose refinement after detection: 1280x1024 scenes with
a 200x200 part (about 2000 edge points), poses perturbed from ground truth by
up to 1.5 px and 1.5 degrees, plus poses at the image border and outside it.
"""

import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402

# FP32 score tolerance (absolute), as for the integer-pose scorer
TOL_SCORE = 1e-5
# FP32 derivative tolerance (absolute) where no sample is near a cell border
TOL_GRAD = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()


@pytest.fixture(scope="module")
def scenes():
    tmpl, imgs, triples = synth.config4_triples(n=512)
    model = sam.Model(tmpl, 30, 60, 4, 1.0)
    om = oracle.create_model(tmpl, 30, 60, 4, 1.0)
    dimgs = [torch.from_numpy(im).cuda() for im in imgs]
    fields = [sam.unit_field(d, 30) for d in dimgs]
    ofields = [oracle.search_fields(im, 1, 30)[0] for im in imgs]
    return model, om, fields, ofields, triples, tmpl


def _poses(triples, which="init"):
    sel = [t[2] if which == "init" else t[1] for t in triples]
    p = torch.tensor(sel, dtype=torch.float32).cuda()
    f = torch.tensor([t[0] for t in triples], dtype=torch.int32).cuda()
    return p, f


def _near_bound(om, pts_r, n):
    # largest change of one point's one-sided derivative at a cell border:
    # x, y parts <= 4 (difference of differences of unit vectors), theta part
    # <= (2 + 4 r) pi/180 with r the point's distance from the reference
    return np.array([4.0, 4.0, (2 + 4 * pts_r) * math.pi / 180]) / n


def test_unit_field_matches_oracle(scenes):
    _, _, fields, ofields, _, _ = scenes
    for f, of in zip(fields, ofields):
        assert np.abs(f.cpu().numpy().astype(np.float64) - of).max() < 2e-7


def test_forward_gradient_normal_match_oracle(scenes):
    model, om, fields, ofields, triples, _ = scenes
    pts = om.points[0]
    n = len(pts[0])
    rmax = float(np.max(np.hypot(pts[0], pts[1])))
    poses, pf = _poses(triples[:192])
    s, g, nrm = sam.score_bilinear(model, fields, poses, pf, grad=True, normal=True)
    s, g, nrm = s.cpu().numpy(), g.cpu().numpy(), nrm.cpu().numpy()
    hp = poses.cpu().numpy().astype(np.float64)
    tight = 0
    for b, (k, _, _) in enumerate(triples[:192]):
        x, y, th = hp[b]
        os_, o = oracle.score_bilinear(ofields[k], pts, x, y, th, want=("grad", "jtj", "jtr"))
        assert abs(s[b] - os_) < TOL_SCORE, (b, s[b], os_)
        near = int(oracle.bilinear_border_mask(pts, x, y, th, 1e-4).sum())
        tol = TOL_GRAD + near * _near_bound(om, rmax, n)
        assert (np.abs(g[b] - o["grad"]) <= tol).all(), (b, near, g[b], o["grad"])
        if near == 0:
            tight += 1
            np.testing.assert_allclose(nrm[b, :6], o["jtj"], rtol=0, atol=5e-5)
            np.testing.assert_allclose(nrm[b, 6:], o["jtr"], rtol=0, atol=5e-5)
    assert tight > 20


def test_border_and_outside_poses(scenes):
    # samples falling outside the image count as zero field
    model, om, fields, ofields, _, _ = scenes
    pts = om.points[0]
    H, W = ofields[0].shape[:2]
    cand = [(3.3, 5.7, 10.0), (W - 2.2, H - 3.9, 200.0), (-40.5, 500.25, 33.0), (W + 300.0, H + 300.0, 0.0),
            (640.0, -120.7, 91.0), (0.0, 0.0, 0.0), (W - 1.0, H - 1.0, 359.99)]
    poses = torch.tensor(cand, dtype=torch.float32).cuda()
    s, g = sam.score_bilinear(model, fields[:1], poses, grad=True)
    for b, (x, y, th) in enumerate(poses.cpu().numpy().astype(np.float64)):
        os_, o = oracle.score_bilinear(ofields[0], pts, x, y, th, want=("grad",))
        assert abs(float(s[b]) - os_) < TOL_SCORE
        if not oracle.bilinear_border_mask(pts, x, y, th, 1e-4).any():
            assert np.abs(g[b].cpu().numpy() - o["grad"]).max() < TOL_GRAD
    assert float(s[3]) == 0.0 and not g[3].any()


def test_polarity_ignoring_variant(scenes):
    _, _, fields, ofields, triples, tmpl = scenes
    model1 = sam.Model(tmpl, 30, 60, 4, 1.0, polarity=1)
    om1 = oracle.create_model(tmpl, 30, 60, 4, 1.0, polarity=1)
    pts = om1.points[0]
    poses, pf = _poses(triples[:48])
    s, g = sam.score_bilinear(model1, fields, poses, pf, grad=True)
    hp = poses.cpu().numpy().astype(np.float64)
    for b, (k, _, _) in enumerate(triples[:48]):
        os_, o = oracle.score_bilinear(ofields[k], pts, *hp[b], polarity=1, want=("grad",))
        assert abs(float(s[b]) - os_) < TOL_SCORE
        if not oracle.bilinear_border_mask(pts, *hp[b], 1e-4).any():
            assert np.abs(g[b].cpu().numpy() - o["grad"]).max() < TOL_GRAD


def test_adjoint_and_autograd(scenes):
    model, om, fields, ofields, triples, _ = scenes
    poses, pf = _poses(triples[:256])
    _, g = sam.score_bilinear(model, fields, poses, pf, grad=True)
    w = torch.randn(256, device="cuda")
    adj = sam.score_bilinear_adjoint(model, fields, poses, w, pf)
    torch.testing.assert_close(adj, w[:, None] * g, rtol=1e-6, atol=1e-7)
    p = poses.clone().requires_grad_(True)
    s = sam.bilinear_score(p, model, fields, pf)
    (w * s).sum().backward()
    torch.testing.assert_close(p.grad, adj, rtol=0, atol=0)
    torch.testing.assert_close(s.detach(), sam.score_bilinear(model, fields, poses, pf), rtol=0, atol=0)


def test_central_differences_h1e3(scenes):
    # central differences of the FP32 forward with h = 1e-3 px / deg against
    # the adjoint; allowed gap: FP32 noise of the two scores / 2h, plus the
    # derivative jump of every point whose sample crosses a cell border
    # within the step
    model, om, fields, ofields, triples, _ = scenes
    pts = om.points[0]
    n = len(pts[0])
    r = np.hypot(pts[0], pts[1])
    rmax = float(r.max())
    h = 1e-3
    B = 64
    poses, pf = _poses(triples[:B])
    _, g = sam.score_bilinear(model, fields, poses, pf, grad=True)
    g = g.cpu().numpy()
    hp = poses.cpu().numpy().astype(np.float64)
    for j in range(3):
        dp = torch.zeros_like(poses)
        dp[:, j] = h
        fd = ((sam.score_bilinear(model, fields, poses + dp, pf) - sam.score_bilinear(model, fields, poses - dp, pf))
              .cpu().numpy().astype(np.float64))
        # the FP32 poses +- h as actually evaluated
        step = ((poses + dp)[:, j] - (poses - dp)[:, j]).cpu().numpy().astype(np.float64)
        fd /= step
        for b in range(B):
            reach = h if j < 2 else rmax * math.radians(h)
            near = int(oracle.bilinear_border_mask(pts, *hp[b], reach * 1.01).sum())
            tol = 2 * 2e-7 / (2 * h) + near * _near_bound(om, rmax, n)[j] + 1e-5
            assert abs(fd[b] - g[b, j]) <= tol, (j, b, fd[b], g[b, j], near)


def test_refine_matches_oracle_and_reaches_truth(scenes):
    model, om, fields, ofields, triples, _ = scenes
    pts = om.points[0]
    B = 128
    poses, pf = _poses(triples[:B])
    init = poses.cpu().numpy().astype(np.float64)
    s = sam.refine_poses(model, fields, poses, pf, iterations=20).cpu().numpy()
    got = poses.cpu().numpy().astype(np.float64)
    close, ok_truth = 0, 0
    for b, (k, gt, _) in enumerate(triples[:B]):
        op, os_ = oracle.refine_gn(ofields[k], pts, init[b], iterations=20)
        # the GPU's final score is M_c at its final pose
        assert abs(s[b] - oracle.score_bilinear(ofields[k], pts, *got[b])) < TOL_SCORE
        # both reach the same optimum up to the flatness of the score there
        assert s[b] >= os_ - 2e-4, (b, s[b], os_)
        close += np.abs(got[b] - op).max() < 0.01
        ok_truth += (np.abs(got[b, :2] - gt[:2]).max() < 0.05) and abs(got[b, 2] - gt[2]) < 0.05
    assert close >= 0.9 * B, close
    assert ok_truth >= 0.85 * B, ok_truth


def test_refine_edge_cases(scenes):
    model, om, fields, ofields, triples, _ = scenes
    poses, pf = _poses(triples[:8])
    before = poses.clone()
    s = sam.refine_poses(model, fields, poses, pf, iterations=0)
    assert torch.equal(poses, before)
    torch.testing.assert_close(s, sam.score_bilinear(model, fields, poses, pf), rtol=0, atol=1e-6)
    # bad field index and non-finite pose -> NaN, others untouched
    bad_pf = pf.clone()
    bad_pf[1] = 7
    p2 = before.clone()
    p2[2, 0] = float("nan")
    out = sam.score_bilinear(model, fields, p2, bad_pf)
    assert torch.isnan(out[1]) and torch.isnan(out[2]) and torch.isfinite(out[[0, 3, 4, 5, 6, 7]]).all()
    s3 = sam.refine_poses(model, fields, p2, bad_pf, iterations=5)
    assert torch.isnan(s3[1]) and torch.isnan(s3[2])
    # empty batch is a no-op
    empty = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    assert sam.score_bilinear(model, fields, empty).numel() == 0
    with pytest.raises(sam.SamError):
        sam.score_bilinear(model, fields, poses, level=9)
    with pytest.raises(ValueError):
        sam.score_bilinear(model, [], poses)


def test_pitched_field_views(scenes):
    # a field whose rows are longer than the image (pitch > w)
    model, om, fields, ofields, triples, _ = scenes
    f = fields[0]
    H, W = f.shape[:2]
    big = torch.zeros((H, W + 24, 2), dtype=torch.float32, device="cuda")
    big[:, :W] = f
    view = big[:, :W]
    poses, _ = _poses([t for t in triples if t[0] == 0][:16])
    a = sam.score_bilinear(model, [view], poses)
    b = sam.score_bilinear(model, [f], poses)
    torch.testing.assert_close(a, b, rtol=0, atol=0)

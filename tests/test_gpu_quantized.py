"""GPU parity of the quantised-direction score (sam_score_map_quantized).

Against the FP64 oracle: the response maps within 1e-6 (FP32 dot products of
unit vectors), the score map within 1e-5 on a top level (both polarities,
both neighbourhood sizes), and the documented approximation bound against the
exact Eq. (1) map of the library's own exhaustive scorer.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402
from paper_2112_05576_gb300.sam import SAM_ERR_ARG  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sam.lib()


def _case(polarity):
    tm, sc, _ = synth.config1_scene()
    m = sam.Model(tm, 30, 60, 3, 1.0, polarity)
    om = oracle.create_model(tm, 30, 60, 3, 1.0, polarity)
    top = oracle.pyramid(sc, 3)[2]
    return m, om, top


@pytest.mark.parametrize("nbins,nbhd,polarity", [(16, 3, 0), (8, 1, 0), (16, 3, 1), (32, 3, 0)])
def test_quantized_matches_oracle(nbins, nbhd, polarity):
    m, om, top = _case(polarity)
    h, w = top.shape
    field = sam.unit_field(torch.from_numpy(np.ascontiguousarray(top)).cuda(), 30)
    maps = torch.empty(sam.response_maps_bytes(w, h, nbins), dtype=torch.uint8, device="cuda")
    got = sam.score_map_quantized(m, 2, field, nbins, nbhd, maps=maps).cpu().numpy()
    f = oracle.search_fields(top, 1, 30)[0]
    R = oracle.response_maps(f, nbins, nbhd=nbhd, polarity=polarity)
    Rg = maps.view(torch.float32)[: nbins * (h + 2) * (w + 2)].view(nbins, h + 2, w + 2).cpu().numpy()
    assert np.max(np.abs(Rg - R)) < 1e-6
    ref = oracle.score_map_quantized(f, om.points[2], om.ntheta(2), om.dtheta(2), nbins, nbhd=nbhd,
                                     polarity=polarity)
    assert np.max(np.abs(got - ref)) < 1e-5


def test_quantized_within_bound_of_exact():
    m, om, top = _case(0)
    h, w = top.shape
    field = sam.unit_field(torch.from_numpy(np.ascontiguousarray(top)).cuda(), 30)
    q = sam.score_map_quantized(m, 2, field, 16, 3).cpu().numpy()
    pf = torch.zeros((h, sam.field_pitch(w, sam.LAYOUT_PAIRS), 2), dtype=torch.float32, device="cuda")
    sam.gradient(torch.from_numpy(np.ascontiguousarray(top)).cuda(), 30, sam.FP32, pf, layout=sam.LAYOUT_PAIRS)
    exact = torch.empty((m.num_angles(2), h, w), dtype=torch.float32, device="cuda")
    sam.score_map(m, 2, pf, w, h, sam.FP32, exact, 1, 1, 3, 0.0, 0, layout=sam.LAYOUT_PAIRS)
    err = np.abs(q - exact.cpu().numpy())
    assert err.max() <= 2 * np.sin(2 * np.pi / 16 / 4) + 1e-5


def test_quantized_rejects_bad_args():
    m, _, top = _case(0)
    h, w = top.shape
    field = sam.unit_field(torch.from_numpy(np.ascontiguousarray(top)).cuda(), 30)
    for nbins in (1, 65):
        with pytest.raises(sam.SamError) as e:
            sam.score_map_quantized(m, 2, field, nbins, 3, maps=torch.empty(16, dtype=torch.uint8, device="cuda"))
        assert e.value.status == SAM_ERR_ARG
    with pytest.raises(sam.SamError) as e:   # scratch too small
        sam.score_map_quantized(m, 2, field, 16, 3, maps=torch.empty(64, dtype=torch.uint8, device="cuda"))
    assert e.value.status == SAM_ERR_ARG

"""Pins of the oracle's quantised-direction form (response maps; an
approximation of Eq. (1) that replaces each rotated model direction by the
centre of its orientation bin).

Pinned against what the mathematics fixes:
- the approximation bound: a vote is 1-Lipschitz in the direction (|w_hat|
  <= 1), and a direction is at most half a bin from its centre, so
  |M_q - M| <= 2 sin(bin width / 4) for every pose; with many bins M_q -> M;
- the response-map decomposition: the quantised score is the mean of the
  precomputed window maxima R_b at the projected points (an independent
  numpy sum over the maps), and every map equals the brute-force
  maximum filter of u_b . w_hat with zeros outside the image;
- bin rule: bin centres map to themselves, opposite directions share a bin
  with polarity 1, and random directions agree with numpy's arctan2.
"""

import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth


@pytest.fixture(scope="module")
def small():
    tm, sc, _ = synth.config1_scene()
    om = oracle.create_model(tm, 30, 60, 3, 1.0)   # top level: 90 angles of 4 degrees
    top = oracle.pyramid(sc, 3)[2]
    f = oracle.search_fields(top, 1, 30)[0]
    return om, f


@pytest.mark.parametrize("nbins,polarity", [(16, 0), (8, 0), (16, 1), (1024, 0), (1024, 1)])
def test_approximation_bound(small, nbins, polarity):
    om, f = small
    nth = om.ntheta(2)
    exact = oracle.score_map(f, om.points[2], nth, om.dtheta(2), nbhd=3, polarity=polarity)
    q = oracle.score_map_quantized(f, om.points[2], nth, om.dtheta(2), nbins, nbhd=3, polarity=polarity)
    width = (np.pi if polarity else 2 * np.pi) / nbins
    err = np.max(np.abs(q - exact))
    assert err <= 2 * np.sin(width / 4) + 1e-12
    if nbins >= 1024:
        assert err < 1e-2


@pytest.mark.parametrize("polarity", [0, 1])
def test_response_maps_are_window_maxima(small, polarity):
    om, f = small
    h, w = f.shape[:2]
    nbins = 16
    R = oracle.response_maps(f, nbins, nbhd=3, polarity=polarity)
    pad = np.zeros((h + 2, w + 2, 2))
    pad[1:-1, 1:-1] = f
    for b in range(nbins):
        phi = b * (np.pi if polarity else 2 * np.pi) / nbins
        dots = np.cos(phi) * pad[..., 0] + np.sin(phi) * pad[..., 1]
        if polarity:
            dots = np.abs(dots)
        # window maxima over the padded image; a window reaching beyond the
        # pad sees zeros as well
        want = ndimage.maximum_filter(dots, size=3, mode="constant", cval=0.0)
        assert np.allclose(R[b], want, atol=1e-15)


@pytest.mark.parametrize("polarity", [0, 1])
def test_score_is_mean_of_response_maps(small, polarity):
    om, f = small
    h, w = f.shape[:2]
    nbins, nth = 16, om.ntheta(2)
    R = oracle.response_maps(f, nbins, nbhd=3, polarity=polarity)
    q = oracle.score_map_quantized(f, om.points[2], nth, om.dtheta(2), nbins, nbhd=3, polarity=polarity)
    for k in (0, 7, nth // 2):
        ox, oy, px, py = oracle.rotate_points(om.points[2], k, om.dtheta(2))
        bins = [oracle.quant_bin(a, b_, nbins, polarity) for a, b_ in zip(px, py)]
        want = np.zeros((h, w))
        for i in range(len(ox)):
            ys, xs = np.arange(h) + oy[i], np.arange(w) + ox[i]
            yy, xx = np.meshgrid(ys, xs, indexing="ij")
            inside = (yy >= -1) & (yy <= h) & (xx >= -1) & (xx <= w)
            v = np.zeros((h, w))
            v[inside] = R[bins[i], yy[inside] + 1, xx[inside] + 1]
            want += v
        assert np.allclose(q[k], want / len(ox), atol=1e-12)


def test_bin_rule():
    for nbins in (8, 16, 32):
        for b in range(nbins):
            phi = 2 * np.pi * b / nbins
            assert oracle.quant_bin(np.cos(phi), np.sin(phi), nbins) == b
            phi1 = np.pi * b / nbins
            assert oracle.quant_bin(np.cos(phi1), np.sin(phi1), nbins, 1) == b
            assert oracle.quant_bin(-np.cos(phi1), -np.sin(phi1), nbins, 1) == b
    rng = np.random.default_rng(3)
    for a in rng.uniform(-np.pi, np.pi, 500):
        want = int(np.floor(a / (2 * np.pi / 16) + 0.5)) % 16
        assert oracle.quant_bin(np.cos(a), np.sin(a), 16) == want

"""Pins of the oracle's angle-only 16-bit storage form.

An edge pixel of the search image is stored as 0x8000 | a, a the direction
atan2(gy, gx) rounded to 2^15 steps of 2 pi / 32768; other pixels as 0.
What fixes it, independently of the oracle's own code:
  * axis and diagonal gradients land on exact multiples of 8192 / 4096;
  * the edge rule is the search threshold, exact at the boundary;
  * rotating the gradient by 90 or 180 degrees or mirroring it shifts or
    negates a exactly, over every gradient a 3x3 Sobel can produce (this
    needs the code to be well defined: no atan2 value lies within 1e-6
    steps of a rounding boundary, checked with numpy's arctan2);
  * the decoded unit vector is within 2 sin(pi / 65536) of g / |g| (half a
    step), and that bound is nearly reached (so the step is 2 pi / 32768);
  * Eq. (1) scores from the decoded field stay within the same bound of the
    exact field's scores.
"""

import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

CHORD = 2.0 * math.sin(math.pi / 65536.0)   # half a step, as a chord
LOW = 30


@pytest.fixture(scope="module")
def all_gradients():
    r = np.arange(-1020, 1021, dtype=np.int32)      # the range of a 3x3 Sobel on uint8
    gx, gy = np.meshgrid(r, r)
    return gx, gy


def test_axis_and_diagonal_codes():
    gx = np.array([200, 0, -200, 0, 200, -200, -200, 200], np.int32)
    gy = np.array([0, 200, 0, -200, 200, 200, -200, -200], np.int32)
    want = [0, 8192, 16384, 24576, 4096, 12288, 20480, 28672]
    assert (oracle.angle_codes(gx, gy, LOW) == np.array(want) + 0x8000).all()
    f = oracle.angle_field(oracle.angle_codes(gx, gy, LOW))
    g = np.stack([gx, gy], 1) / np.hypot(gx, gy)[:, None]
    assert np.abs(f - g).max() < 1e-15


def test_edge_threshold_is_the_search_rule():
    # gx^2 + gy^2 >= 16 low^2: (120, 0) and (72, 96) sit exactly on it
    gx = np.array([120, 119, 72, 72, 0, 0], np.int32)
    gy = np.array([0, 0, 96, 95, 0, 120], np.int32)
    c = oracle.angle_codes(gx, gy, LOW)
    assert [(v >> 15) for v in c] == [1, 0, 1, 0, 0, 1]
    assert (oracle.angle_field(c)[[1, 3, 4]] == 0).all()


def test_codes_are_well_defined_and_exactly_equivariant(all_gradients):
    gx, gy = all_gradients
    t = np.arctan2(gy.astype(np.float64), gx) * (32768 / (2 * np.pi))
    edge = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2 >= 16 * LOW * LOW
    frac = t[edge] - np.floor(t[edge])
    assert np.abs(frac - 0.5).min() > 1e-6
    a = oracle.angle_codes(gx, gy, LOW).astype(np.int64)
    assert ((a >> 15) == edge).all()
    a = a & 0x7fff
    rot90 = oracle.angle_codes(-gy, gx, LOW).astype(np.int64) & 0x7fff       # +90 degrees
    rot180 = oracle.angle_codes(-gx, -gy, LOW).astype(np.int64) & 0x7fff
    mirror = oracle.angle_codes(gx, -gy, LOW).astype(np.int64) & 0x7fff      # angle -> -angle
    assert (rot90[edge] == (a[edge] + 8192) % 32768).all()
    assert (rot180[edge] == (a[edge] + 16384) % 32768).all()
    assert (mirror[edge] == (-a[edge]) % 32768).all()


def test_decoded_direction_within_half_a_step(all_gradients):
    gx, gy = all_gradients
    f = oracle.angle_field(oracle.angle_codes(gx, gy, LOW))
    edge = gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2 >= 16 * LOW * LOW
    m = np.hypot(gx, gy)
    err = np.hypot(f[..., 0] - gx / np.where(m > 0, m, 1), f[..., 1] - gy / np.where(m > 0, m, 1))[edge]
    assert err.max() <= CHORD + 1e-15
    assert err.max() > 0.95 * CHORD      # the step is 2 pi / 32768, not finer
    assert (np.abs(np.hypot(f[..., 0], f[..., 1])[edge] - 1.0) < 1e-15).all()
    assert (f[~edge] == 0).all()


@pytest.mark.parametrize("polarity", [0, 1])
def test_scores_within_the_storage_bound(polarity):
    tmpl, img, truth = synth.config1_scene()
    om = oracle.create_model(tmpl, 30, 60, 3, 1.0)
    top = 2
    exact = oracle.search_fields(img, 3, LOW)[top]
    codes, dec = oracle.search_angle_fields(img, 3, LOW)[top]
    assert ((codes != 0) == np.any(exact != 0, axis=2)).all()
    nth, dth = om.ntheta(top), om.dtheta(top)
    m_exact = oracle.score_map(exact, om.points[top], nth, dth, polarity=polarity)
    m_code = oracle.score_map(dec, om.points[top], nth, dth, polarity=polarity)
    d = np.abs(m_code - m_exact)
    assert d.max() <= CHORD + 1e-12
    assert d.max() > 0.0
    # the best pose is an instance's in both
    assert np.unravel_index(np.argmax(m_code), m_code.shape) == np.unravel_index(np.argmax(m_exact), m_exact.shape)

"""ctypes marshalling and step composition for the C oracle.

TEST INFRASTRUCTURE: see the package docstring.  Every function here either
calls one C routine of ``sam_oracle.c`` or composes them in the order of
Sec. II of the paper (edge extraction -> pyramid -> top-level exhaustive
search -> refinement down the pyramid -> best poses).
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sam_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsam_oracle.so")
_lib = None

_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_c_int = ctypes.c_int
_c_dbl = ctypes.c_double
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile sam_oracle.c into a shared library (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.or_pyramid_down.argtypes = [_u8p, _c_int, _c_int, _u8p]
        lib.or_sobel.argtypes = [_u8p, _c_int, _c_int, _i32p, _i32p]
        lib.or_search_mask.argtypes = [_i32p, _i32p, _c_int, _c_int, _u8p]
        lib.or_hysteresis.argtypes = [_i32p, _i32p, _c_int, _c_int, _c_int, _c_int, _u8p]
        lib.or_unit_field.argtypes = [_i32p, _i32p, _u8p, _c_int, _f64p]
        lib.or_model_points.argtypes = [_u8p, _c_int, _c_int, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p]
        lib.or_model_points.restype = _c_int
        lib.or_rotate_points.argtypes = [_i32p, _i32p, _i32p, _i32p, _c_int, _c_int, _c_dbl,
                                         _i32p, _i32p, _f64p, _f64p]
        lib.or_score_pose.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _f64p, _f64p, _c_int,
                                      _c_int, _c_int, _c_int, _c_int]
        lib.or_score_pose.restype = _c_dbl
        lib.or_score_map.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _c_int,
                                     _c_dbl, _c_int, _c_int, _c_int, _c_int, _f64p]
        lib.or_score_map_range.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _c_int,
                                           _c_int, _c_dbl, _c_int, _c_int, _c_int, _c_int, _f64p]
        lib.or_candidates.argtypes = [_f64p, _c_int, _c_int, _c_int, _c_dbl, _c_int, _i32p, _i32p, _i32p, _f64p]
        lib.or_candidates.restype = _c_int
        lib.or_child_shift.argtypes = [_c_int, _c_dbl, _c_dbl, _c_dbl, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]
        lib.or_refine_level.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _c_int,
                                        _c_dbl, _c_dbl, _c_dbl, _c_int, _c_int, _c_dbl, _c_int,
                                        _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _f64p]
        lib.or_nms.argtypes = [_c_int, _i32p, _i32p, _i32p, _f64p, _c_int, _c_int, _c_int, _c_int, _i32p]
        lib.or_nms.restype = _c_int
        lib.or_score_bilinear.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int,
                                          _c_dbl, _c_dbl, _c_dbl, _c_int, _vp, _vp, _vp]
        lib.or_score_bilinear.restype = _c_dbl
        lib.or_bilinear_border_mask.argtypes = [_i32p, _i32p, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _u8p]
        lib.or_bilinear_border_mask.restype = _c_int
        lib.or_refine_gn.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _c_int,
                                     _f64p, _c_int]
        lib.or_refine_gn.restype = _c_dbl
        lib.or_subpixel_fit.argtypes = [_f64p, _f64p]
        lib.or_quant_bin.argtypes = [_c_dbl, _c_dbl, _c_int, _c_int]
        lib.or_quant_bin.restype = _c_int
        lib.or_score_map_quantized.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _c_int,
                                               _c_dbl, _c_int, _c_int, _c_int, _f64p]
        lib.or_response_maps.argtypes = [_f64p, _c_int, _c_int, _c_int, _c_int, _c_int, _f64p]
        lib.or_angle_codes.argtypes = [_i32p, _i32p, _c_int, _c_int, _u16p]
        lib.or_angle_field.argtypes = [_u16p, _c_int, _f64p]
        lib.or_project_affine.argtypes = [_i32p, _i32p, _i32p, _i32p, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl,
                                          _i32p, _i32p, _f64p, _f64p]
        lib.or_project_affine.restype = _c_int
        lib.or_scaled_points.argtypes = [_i32p, _i32p, _i32p, _i32p, _c_int, _c_int, _c_dbl, _c_dbl,
                                         _i32p, _i32p, _f64p, _f64p]
        lib.or_scaled_points.restype = _c_int
        lib.or_score_map_scaled.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _f64p, _c_int,
                                            _c_int, _c_dbl, _c_int, _c_int, _f64p]
        lib.or_candidates_scaled.argtypes = [_f64p, _c_int, _c_int, _c_int, _c_int, _c_dbl, _c_int, _i32p, _i32p,
                                             _i32p, _i32p, _f64p]
        lib.or_candidates_scaled.restype = _c_int
        lib.or_child_shift_scaled.argtypes = [_c_int, _c_dbl, _c_dbl, _c_dbl, _c_dbl, ctypes.POINTER(ctypes.c_int32),
                                              ctypes.POINTER(ctypes.c_int32)]
        lib.or_refine_level_scaled.argtypes = [_f64p, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _c_int, _f64p,
                                               _c_int, _c_int, _c_dbl, _c_dbl, _c_dbl, _c_int, _c_int, _c_dbl, _c_int,
                                               _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _i32p, _f64p]
        _lib = lib
    return _lib


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# edge extraction and pyramid (Sec. II)
# ---------------------------------------------------------------------------

def pyramid_down(img):
    """One pyramid step (Sec. II image pyramid, of intensities): 2x2 mean rounded half up, odd row/column
    dropped."""
    img = _u8(img)
    h, w = img.shape
    out = np.empty((h // 2, w // 2), dtype=np.uint8)
    _L().or_pyramid_down(img, w, h, out)
    return out


def pyramid(img, levels):
    """The intensity pyramid (Sec. II), level 0 first."""
    out = [_u8(img)]
    for _ in range(1, levels):
        out.append(pyramid_down(out[-1]))
    return out


def sobel(img):
    """Integer 3x3 Sobel gx, gy (Sec. II x- and y-gradients; x right, y down), zero on the 1-pixel border."""
    img = _u8(img)
    h, w = img.shape
    gx = np.empty((h, w), dtype=np.int32)
    gy = np.empty((h, w), dtype=np.int32)
    _L().or_sobel(img, w, h, gx, gy)
    return gx, gy


def search_mask(gx, gy, low):
    """Search-image edges (Sec. II edge thresholds, magnitude |g|/4): gx^2 + gy^2 >= 16 low^2."""
    gx, gy = _i32(gx), _i32(gy)
    m = np.empty(gx.shape, dtype=np.uint8)
    _L().or_search_mask(gx, gy, gx.size, int(low), m)
    return m


def hysteresis(gx, gy, low, high):
    """Model edges (Sec. II edge thresholds, magnitude |g|/4): >= high seeds grown 8-connected through >= low."""
    gx, gy = _i32(gx), _i32(gy)
    h, w = gx.shape
    m = np.empty(gx.shape, dtype=np.uint8)
    _L().or_hysteresis(gx, gy, w, h, int(low), int(high), m)
    return m


def unit_field(gx, gy, mask):
    """The unit field g/|g| on edges, (0, 0) elsewhere (the normalised gradients of Eq. (1))."""
    gx, gy, mask = _i32(gx), _i32(gy), _u8(mask)
    f = np.empty(gx.shape + (2,), dtype=np.float64)
    _L().or_unit_field(gx, gy, mask, gx.size, f)
    return f


def model_points(tmpl, low, high):
    """(tx, ty, gx, gy) int32 arrays of one template level's edge points."""
    tmpl = _u8(tmpl)
    h, w = tmpl.shape
    tx, ty, gx, gy = (np.empty(w * h, dtype=np.int32) for _ in range(4))
    n = _L().or_model_points(tmpl, w, h, int(low), int(high), tx, ty, gx, gy)
    return tx[:n].copy(), ty[:n].copy(), gx[:n].copy(), gy[:n].copy()


@dataclass
class OracleModel:
    """Template pyramid and per-level edge points (Sec. II inputs)."""

    levels: int
    angle_step_deg: float           # at level 0
    low: int
    high: int
    polarity: int
    sizes: list = field(default_factory=list)     # (w, h) per level
    points: list = field(default_factory=list)    # (tx, ty, gx, gy) per level

    def ntheta(self, level):
        return int(round(360.0 / self.angle_step_deg)) >> level

    def dtheta(self, level):
        return self.angle_step_deg * (2 ** level)


def create_model(tmpl, low, high, levels, angle_step_deg, polarity=0):
    """The model of Sec. II: template pyramid and per-level edge points (t, g)."""
    n0 = int(round(360.0 / angle_step_deg))
    if abs(n0 * angle_step_deg - 360.0) > 1e-9 or n0 % (1 << (levels - 1)) != 0:
        raise ValueError("360 / angle_step must be an integer divisible by 2^(levels-1)")
    m = OracleModel(levels=levels, angle_step_deg=float(angle_step_deg), low=low, high=high, polarity=polarity)
    for lvl, img in enumerate(pyramid(tmpl, levels)):
        m.sizes.append((img.shape[1], img.shape[0]))
        pts = model_points(img, low, high)
        if len(pts[0]) == 0:
            raise ValueError(f"template level {lvl} has no edge points")
        m.points.append(pts)
    return m


def search_fields(img, levels, low):
    """Per-level FP64 unit gradient fields of the search image (H x W x 2)."""
    out = []
    for lvl_img in pyramid(img, levels):
        gx, gy = sobel(lvl_img)
        out.append(unit_field(gx, gy, search_mask(gx, gy, low)))
    return out


# ---------------------------------------------------------------------------
# scoring (Eq. (1), Eq. (2), neighbouring search)
# ---------------------------------------------------------------------------

def rotate_points(pts, k, dtheta_deg):
    """Eq. (2) for angle index k: integer offsets floor(R(theta) t + 1/2) in FP64 and the model gradients
    turned by the same R(theta), as unit directions."""
    tx, ty, gx, gy = pts
    n = len(tx)
    ox, oy = np.empty(n, np.int32), np.empty(n, np.int32)
    px, py = np.empty(n, np.float64), np.empty(n, np.float64)
    _L().or_rotate_points(tx, ty, gx, gy, n, int(k), float(dtheta_deg), ox, oy, px, py)
    return ox, oy, px, py


def score_pose(field, rot, ux, uy, nbhd=3, polarity=0):
    """Eq. (1) at one pose with the neighbouring search of size nbhd (Fig. 3): per point the best vote over
    its window of p . w (|p . w| with polarity 1), 0 outside the image and on non-edge pixels."""
    field = _f64(field)
    h, w = field.shape[:2]
    ox, oy, px, py = rot
    return _L().or_score_pose(field, w, h, ox, oy, px, py, len(ox), int(ux), int(uy), int(nbhd), int(polarity))


def score_map(field, pts, ntheta, dtheta_deg, step_x=1, step_y=1, nbhd=3, polarity=0):
    """Exhaustive map M[k, gy, gx] over all poses of the step grid."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = (_i32(a) for a in pts)
    gw, gh = (w + step_x - 1) // step_x, (h + step_y - 1) // step_y
    out = np.empty((ntheta, gh, gw), dtype=np.float64)
    _L().or_score_map(field, w, h, tx, ty, gx, gy, len(tx), int(ntheta), float(dtheta_deg), int(step_x),
                      int(step_y), int(nbhd), int(polarity), out)
    return out


def score_map_range(field, pts, k_begin, k_count, dtheta_deg, step_x=1, step_y=1, nbhd=3, polarity=0):
    """Slice [k_begin, k_begin + k_count) of the exhaustive map."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = (_i32(a) for a in pts)
    gw, gh = (w + step_x - 1) // step_x, (h + step_y - 1) // step_y
    out = np.empty((k_count, gh, gw), dtype=np.float64)
    _L().or_score_map_range(field, w, h, tx, ty, gx, gy, len(tx), int(k_begin), int(k_count), float(dtheta_deg),
                            int(step_x), int(step_y), int(nbhd), int(polarity), out)
    return out


def candidates(smap, min_score, K):
    """Top-K strict 3x3x3 local maxima (theta circular) with M >= min_score.

    Returns arrays (k, gy, gx, score) sorted best first.
    """
    smap = _f64(smap)
    nth, gh, gw = smap.shape
    ck, cy, cx = (np.empty(K, np.int32) for _ in range(3))
    cs = np.empty(K, np.float64)
    n = _L().or_candidates(smap, nth, gh, gw, float(min_score), int(K), ck, cy, cx, cs)
    return ck[:n].copy(), cy[:n].copy(), cx[:n].copy(), cs[:n].copy()


def _ref_shift_d(model, level):
    """d = 2 c_{l+1} + 1/2 - c_l per axis for the step from level+1 to level."""
    (w0, h0), (w1, h1) = model.sizes[level], model.sizes[level + 1]
    return 2 * (w1 // 2) + 0.5 - (w0 // 2), 2 * (h1 // 2) + 0.5 - (h0 // 2)


def child_shift(model, level, k_parent):
    """Coarse-to-fine child shift of a level+1 parent with angle index k_parent: its level-`level` centre is
    2 (x, y) + shift (the reference-point offset between levels, turned by the parent's angle)."""
    dx, dy = _ref_shift_d(model, level)
    sx, sy = ctypes.c_int32(), ctypes.c_int32()
    _L().or_child_shift(int(k_parent), float(model.dtheta(level + 1)), dx, dy, ctypes.byref(sx), ctypes.byref(sy))
    return sx.value, sy.value


def refine_level(model, level, field, xs, ys, ks, nbhd, polarity, min_score):
    """Best of the 27 level-`level` poses around each level+1 parent pose."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = model.points[level]
    n = len(xs)
    ox, oy, ok = (np.empty(n, np.int32) for _ in range(3))
    os_ = np.empty(n, np.float64)
    dx, dy = _ref_shift_d(model, level)
    _L().or_refine_level(field, w, h, tx, ty, gx, gy, len(tx), model.ntheta(level), float(model.dtheta(level)),
                         dx, dy, int(nbhd), int(polarity), float(min_score), n,
                         _i32(xs), _i32(ys), _i32(ks), ox, oy, ok, os_)
    return ox, oy, ok, os_


def nms(xs, ys, ks, ss, w, h, min_side, max_out):
    """Final non-maximum suppression: greedy by score (ties: smaller (k, y, x) key), dropping poses closer
    than half the smaller template side to a kept one."""
    n = len(xs)
    keep = np.empty(max(n, 1), np.int32)
    nk = _L().or_nms(n, _i32(xs), _i32(ys), _i32(ks), _f64(ss), int(w), int(h), int(min_side), int(max_out), keep)
    return keep[:nk].copy()


@dataclass
class DetectParams:
    step_x: int = 1
    step_y: int = 1
    nbhd: int = 3
    min_score: float = 0.7
    max_detections: int = 16
    top_k: int = 64


def detect(model: OracleModel, img, params: DetectParams, trace=None):
    """Full detection, Sec. II order.

    Returns a list of (x, y, theta_deg, score, k) at level 0, best first.
    If `trace` is a dict it receives the intermediate results per level.
    """
    L = model.levels
    fields = search_fields(img, L, model.low)
    top = L - 1
    smap = score_map(fields[top], model.points[top], model.ntheta(top), model.dtheta(top),
                     params.step_x, params.step_y, params.nbhd, model.polarity)
    ck, cy, cx, cs = candidates(smap, params.min_score, params.top_k)
    xs, ys, ks, ss = cx * params.step_x, cy * params.step_y, ck, cs
    if trace is not None:
        trace["fields"] = fields
        trace["map"] = smap
        trace["cand"] = (xs.copy(), ys.copy(), ks.copy(), ss.copy())
        trace["levels"] = {}
    for lvl in range(top - 1, -1, -1):
        alive = np.isfinite(ss)
        xs, ys, ks, ss = xs[alive], ys[alive], ks[alive], ss[alive]
        xs, ys, ks, ss = refine_level(model, lvl, fields[lvl], xs, ys, ks, params.nbhd, model.polarity,
                                      params.min_score)
        if trace is not None:
            trace["levels"][lvl] = (xs.copy(), ys.copy(), ks.copy(), ss.copy())
    w0, h0 = model.sizes[0]
    H, W = img.shape
    keep = nms(xs, ys, ks, ss, W, H, min(w0, h0), params.max_detections)
    return [(int(xs[i]), int(ys[i]), float(ks[i]) * model.angle_step_deg, float(ss[i]), int(ks[i])) for i in keep]


# ---------------------------------------------------------------------------
# differentiable score on a continuous pose (extension of Eq. (1), Eq. (2))
# ---------------------------------------------------------------------------

def _opt_out(k):
    a = np.zeros(k, dtype=np.float64)
    return a, a.ctypes.data_as(_vp)


def score_bilinear(field, pts, x, y, theta_deg, polarity=0, want=()):
    """M_c at a continuous pose, FP64.  `want` may hold "grad", "jtj", "jtr";
    returns the score alone, or (score, {name: array}) when `want` is set."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = (_i32(a) for a in pts)
    outs = {k: _opt_out(n) for k, n in (("grad", 3), ("jtj", 6), ("jtr", 3)) if k in want}
    ptr = lambda k: outs[k][1] if k in outs else None  # noqa: E731
    s = _L().or_score_bilinear(field, w, h, tx, ty, gx, gy, len(tx), float(x), float(y), float(theta_deg),
                               int(polarity), ptr("grad"), ptr("jtj"), ptr("jtr"))
    if not want:
        return s
    return s, {k: v[0] for k, v in outs.items()}


def bilinear_border_mask(pts, x, y, theta_deg, eps):
    """Boolean mask of the points whose sample lies within eps of a pixel-cell border."""
    tx, ty = _i32(pts[0]), _i32(pts[1])
    mask = np.zeros(len(tx), dtype=np.uint8)
    _L().or_bilinear_border_mask(tx, ty, len(tx), float(x), float(y), float(theta_deg), float(eps), mask)
    return mask.astype(bool)


def refine_gn(field, pts, pose, iterations=20, polarity=0):
    """Damped Gauss-Newton refinement of a continuous pose; returns (pose, M_c)."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = (_i32(a) for a in pts)
    p = np.array(pose, dtype=np.float64)
    s = _L().or_refine_gn(field, w, h, tx, ty, gx, gy, len(tx), int(polarity), p, int(iterations))
    return p, s


# ---------------------------------------------------------------------------
# sub-pixel / sub-angle final pose (quadratic fit of the 3x3x3 neighbourhood)
# ---------------------------------------------------------------------------

def subpixel_fit(s27):
    """(dx, dy, dk) of the quadratic fit of a 3x3x3 score neighbourhood,
    s27[(dk + 1) * 9 + (dy + 1) * 3 + (dx + 1)]; see or_subpixel_fit."""
    s = _f64(np.asarray(s27, dtype=np.float64).reshape(27))
    d = np.zeros(3, dtype=np.float64)
    _L().or_subpixel_fit(s, d)
    return d


def neighbourhood27(field, pts, x, y, k, ntheta, dtheta_deg, nbhd=3, polarity=0):
    """Eq. (1) scores of the 27 poses (x + dx, y + dy, k + dk), dx, dy, dk in
    {-1, 0, 1}, angle index circular; layout of subpixel_fit."""
    out = np.empty(27, dtype=np.float64)
    for dk in (-1, 0, 1):
        rot = rotate_points(pts, (k + dk) % ntheta, dtheta_deg)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out[(dk + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = score_pose(field, rot, x + dx, y + dy, nbhd, polarity)
    return out


def climb27(s27):
    """Index of the neighbour to move to, or 13 (the centre) when no
    neighbour scores strictly higher; among equal best neighbours the first
    in (dk, dy, dx) order."""
    best, j = s27[13], 13
    for i in range(27):
        if s27[i] > best:
            best, j = s27[i], i
    return j


def subpixel_poses(field, pts, kyx, ntheta, dtheta_deg, nbhd=3, polarity=0, max_moves=8):
    """Sub-pixel poses of integer level-0 poses kyx[i] = (k, y, x).  The pose
    first moves to the best of its 27 neighbours until no neighbour scores
    higher (at most max_moves moves; the coarse-to-fine search can stop at
    the edge of its window), then takes the quadratic fit of the
    neighbourhood: rows (x + dx, y + dy, ((k + dk) * dtheta) mod 360,
    M(x, y, k)) at the final integer pose."""
    res = []
    for k, y, x in kyx:
        k, y, x = int(k), int(y), int(x)
        for move in range(max_moves + 1):
            s = neighbourhood27(field, pts, x, y, k, ntheta, dtheta_deg, nbhd, polarity)
            j = climb27(s)
            if j == 13 or move == max_moves:
                break
            k = (k + j // 9 - 1) % ntheta
            y += (j // 3) % 3 - 1
            x += j % 3 - 1
        d = subpixel_fit(s)
        res.append((x + d[0], y + d[1], ((k + d[2]) * dtheta_deg) % 360.0, s[13]))
    return np.array(res, dtype=np.float64).reshape(-1, 4)


# ---------------------------------------------------------------------------
# quantised-direction form (response maps; an approximation of Eq. (1))
# ---------------------------------------------------------------------------

def quant_bin(px, py, nbins, polarity=0):
    """Orientation bin of a unit direction for the quantised-direction form: the nearest of nbins centres
    b 2 pi / nbins (pi / nbins with polarity 1), by FP64 atan2."""
    return int(_L().or_quant_bin(float(px), float(py), int(nbins), int(polarity)))


def score_map_quantized(field, pts, ntheta, dtheta_deg, nbins, nbhd=3, polarity=0):
    """M_q over the full step-1 pose grid: Eq. (1) with each rotated model
    direction replaced by its bin centre; out[k, y, x]."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = (_i32(a) for a in pts)
    out = np.empty((ntheta, h, w), dtype=np.float64)
    _L().or_score_map_quantized(field, w, h, tx, ty, gx, gy, len(tx), int(ntheta), float(dtheta_deg), int(nbins),
                                int(nbhd), int(polarity), out)
    return out


def response_maps(field, nbins, nbhd=3, polarity=0):
    """R[b, y + 1, x + 1] = max over the window at (x, y) of u_b . w_hat, for
    -1 <= x <= w, -1 <= y <= h."""
    field = _f64(field)
    h, w = field.shape[:2]
    out = np.empty((nbins, h + 2, w + 2), dtype=np.float64)
    _L().or_response_maps(field, w, h, int(nbhd), int(polarity), int(nbins), out)
    return out


# ---------------------------------------------------------------------------
# angle-only 16-bit storage of the search field
# ---------------------------------------------------------------------------

def angle_codes(gx, gy, low):
    """uint16 codes: 0x8000 | round(atan2(gy, gx) 32768 / 2 pi) mod 32768 on
    search edges (gx^2 + gy^2 >= 16 low^2), 0 elsewhere."""
    gx, gy = _i32(gx), _i32(gy)
    out = np.empty(gx.shape, dtype=np.uint16)
    _L().or_angle_codes(gx.ravel(), gy.ravel(), gx.size, int(low), out.reshape(-1))
    return out


def angle_field(codes):
    """The FP64 unit field (H x W x 2) the codes stand for."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    out = np.empty(codes.shape + (2,), dtype=np.float64)
    _L().or_angle_field(codes.reshape(-1), codes.size, out.reshape(-1))
    return out


def search_angle_fields(img, levels, low):
    """Per-level angle codes of the search image and the fields they decode to."""
    out = []
    for lvl_img in pyramid(img, levels):
        gx, gy = sobel(lvl_img)
        c = angle_codes(gx, gy, low)
        out.append((c, angle_field(c)))
    return out


# ---------------------------------------------------------------------------
# affine (scaled) poses: a generalisation of Eq. (2)
# ---------------------------------------------------------------------------

def project_affine(pts, A):
    """Eq. (2) with the rotation replaced by a 2x2 matrix A (A = s R(theta) for a
    scaled pose): offsets floor(A t + 1/2), directions A^-T g normalised (the
    gradient of the warped image).  Returns (ox, oy, px, py) like rotate_points."""
    tx, ty, gx, gy = (_i32(a) for a in pts)
    A = np.asarray(A, dtype=np.float64)
    n = len(tx)
    ox, oy = np.empty(n, np.int32), np.empty(n, np.int32)
    px, py = np.empty(n, np.float64), np.empty(n, np.float64)
    if not _L().or_project_affine(tx, ty, gx, gy, n, float(A[0, 0]), float(A[0, 1]), float(A[1, 0]),
                                  float(A[1, 1]), ox, oy, px, py):
        raise ValueError("singular projection matrix")
    return ox, oy, px, py


def similarity(scale, theta_deg):
    """A = scale R(theta) (x right, y down, theta in degrees as in Eq. (2))."""
    th = math.radians(theta_deg)
    c, s = math.cos(th), math.sin(th)
    return np.array([[scale * c, -scale * s], [scale * s, scale * c]])


# ---------------------------------------------------------------------------
# scaled poses: A = s R(theta) over a grid of scales (generalised Eq. (2))
# ---------------------------------------------------------------------------

def scale_grid(scale_min, scale_step, n_scales):
    """s_j = scale_min + j scale_step, j < n_scales (the same grid at every level)."""
    return [float(scale_min) + j * float(scale_step) for j in range(int(n_scales))]


def scaled_points(pts, k, dtheta_deg, scale):
    """Offsets and directions of the model points for scale `scale` and angle
    index k: project_affine with A = scale R(theta_k), the angle computed as
    in rotate_points."""
    tx, ty, gx, gy = (_i32(a) for a in pts)
    n = len(tx)
    ox, oy = np.empty(n, np.int32), np.empty(n, np.int32)
    px, py = np.empty(n, np.float64), np.empty(n, np.float64)
    if not _L().or_scaled_points(tx, ty, gx, gy, n, int(k), float(dtheta_deg), float(scale), ox, oy, px, py):
        raise ValueError("scale 0")
    return ox, oy, px, py


def score_map_scaled(field, pts, scales, ntheta, dtheta_deg, nbhd=3, polarity=0):
    """Exhaustive step-1 map M[j, k, y, x] over scales, angles and translations."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = (_i32(a) for a in pts)
    sc = _f64(scales)
    out = np.empty((len(sc), ntheta, h, w), dtype=np.float64)
    _L().or_score_map_scaled(field, w, h, tx, ty, gx, gy, len(tx), sc, len(sc), int(ntheta), float(dtheta_deg),
                             int(nbhd), int(polarity), out)
    return out


def candidates_scaled(smap, min_score, K):
    """Top-K strict local maxima over (scale, angle circular, y, x) with M >= min_score.

    Returns arrays (j, k, gy, gx, score) sorted best first."""
    smap = _f64(smap)
    ns, nth, gh, gw = smap.shape
    cj, ck, cy, cx = (np.empty(K, np.int32) for _ in range(4))
    cs = np.empty(K, np.float64)
    n = _L().or_candidates_scaled(smap, ns, nth, gh, gw, float(min_score), int(K), cj, ck, cy, cx, cs)
    return cj[:n].copy(), ck[:n].copy(), cy[:n].copy(), cx[:n].copy(), cs[:n].copy()


def child_shift_scaled(model, level, k_parent, scale):
    """child_shift for a parent of scale `scale`."""
    dx, dy = _ref_shift_d(model, level)
    sx, sy = ctypes.c_int32(), ctypes.c_int32()
    _L().or_child_shift_scaled(int(k_parent), float(model.dtheta(level + 1)), float(scale), dx, dy,
                               ctypes.byref(sx), ctypes.byref(sy))
    return sx.value, sy.value


def refine_level_scaled(model, level, field, scales, xs, ys, js, ks, nbhd, polarity, min_score):
    """Best of the up to 81 level-`level` poses (x, y, angle, scale +- 1) around each level+1 parent."""
    field = _f64(field)
    h, w = field.shape[:2]
    tx, ty, gx, gy = model.points[level]
    n = len(xs)
    ox, oy, oj, ok = (np.empty(n, np.int32) for _ in range(4))
    os_ = np.empty(n, np.float64)
    dx, dy = _ref_shift_d(model, level)
    sc = _f64(scales)
    _L().or_refine_level_scaled(field, w, h, tx, ty, gx, gy, len(tx), sc, len(sc), model.ntheta(level),
                                float(model.dtheta(level)), dx, dy, int(nbhd), int(polarity), float(min_score), n,
                                _i32(xs), _i32(ys), _i32(js), _i32(ks), ox, oy, oj, ok, os_)
    return ox, oy, oj, ok, os_


def detect_scaled(model: OracleModel, img, params: DetectParams, scales, trace=None):
    """Full detection over scales, angles and translations, in Sec. II order
    (edge extraction, pyramid, exhaustive top level, refinement down the
    pyramid with the scale searched +- 1 too, NMS keyed by (scale, angle, y,
    x)).  Returns (x, y, theta_deg, score, k, j) at level 0, best first."""
    L = model.levels
    fields = search_fields(img, L, model.low)
    top = L - 1
    smap = score_map_scaled(fields[top], model.points[top], scales, model.ntheta(top), model.dtheta(top),
                            params.nbhd, model.polarity)
    cj, ck, cy, cx, cs = candidates_scaled(smap, params.min_score, params.top_k)
    xs, ys, js, ks, ss = cx, cy, cj, ck, cs
    if trace is not None:
        trace["fields"] = fields
        trace["map"] = smap
        trace["cand"] = (xs.copy(), ys.copy(), js.copy(), ks.copy(), ss.copy())
    for lvl in range(top - 1, -1, -1):
        alive = np.isfinite(ss)
        xs, ys, js, ks, ss = xs[alive], ys[alive], js[alive], ks[alive], ss[alive]
        xs, ys, js, ks, ss = refine_level_scaled(model, lvl, fields[lvl], scales, xs, ys, js, ks, params.nbhd,
                                                 model.polarity, params.min_score)
    w0, h0 = model.sizes[0]
    H, W = img.shape
    nth0 = model.ntheta(0)
    keep = nms(xs, ys, js * nth0 + ks, ss, W, H, min(w0, h0), params.max_detections)
    return [(int(xs[i]), int(ys[i]), float(ks[i]) * model.angle_step_deg, float(ss[i]), int(ks[i]), int(js[i]))
            for i in keep]

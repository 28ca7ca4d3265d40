"""Thin ctypes binding of libsam.so (include/sam.h).

Argument marshalling only: every step of the detector runs in the CUDA
library.  Device buffers are torch CUDA tensors (passed by data pointer) and
the stream is torch's current stream; host buffers are numpy arrays.  If
the library is missing the import of a compute entry point raises: there is
no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import List, Optional

import numpy as np

from . import build as _build

SAM_OK, SAM_ERR_ARG, SAM_ERR_NOMEM, SAM_ERR_CUDA, SAM_ERR_TIMEOUT, SAM_ERR_EMPTY_MODEL, SAM_ERR_CAPACITY = range(7)
FP32, BF16, FP16, ANGLE16 = 0, 1, 2, 3
LAYOUT_PIXEL, LAYOUT_PAIRS = 0, 1

_c_int, _c_float, _c_double, _vp = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_f32p = ctypes.POINTER(ctypes.c_float)


class ModelParams(ctypes.Structure):
    _fields_ = [("low", _c_int), ("high", _c_int), ("levels", _c_int), ("angle_step_deg", _c_double),
                ("polarity", _c_int)]


class DetectParams(ctypes.Structure):
    _fields_ = [("step_x", _c_int), ("step_y", _c_int), ("neighbourhood", _c_int), ("min_score", _c_float),
                ("max_detections", _c_int), ("top_k", _c_int), ("precision", _c_int),
                ("early_termination", _c_int)]


class Pose(ctypes.Structure):
    _fields_ = [("x", _c_float), ("y", _c_float), ("theta_deg", _c_float), ("score", _c_float),
                ("angle_index", _c_int), ("level0_x", _c_int), ("level0_y", _c_int), ("scale_index", _c_int)]


class FieldRef(ctypes.Structure):
    _fields_ = [("field", _vp), ("w", _c_int), ("h", _c_int), ("pitch", _c_int)]


MAX_BILINEAR_FIELDS = 64

# name -> (restype, argtypes); every symbol include/sam.h declares
SIGNATURES = {
    "sam_status_str": (ctypes.c_char_p, [_c_int]),
    "sam_version": (_c_int, []),
    "sam_compiled_arch": (_c_int, []),
    "sam_default_model_params": (None, [ctypes.POINTER(ModelParams)]),
    "sam_default_detect_params": (None, [ctypes.POINTER(DetectParams)]),
    "sam_create_model": (_c_int, [_vp, _c_int, _c_int, _c_int, ctypes.POINTER(ModelParams), ctypes.POINTER(_vp)]),
    "sam_free_model": (None, [_vp]),
    "sam_create_model_scaled": (_c_int, [_vp, _c_int, _c_int, _c_int, ctypes.POINTER(ModelParams), _c_double,
                                         _c_double, _c_int, ctypes.POINTER(_vp)]),
    "sam_model_num_scales": (_c_int, [_vp]),
    "sam_model_scale": (_c_double, [_vp, _c_int]),
    "sam_model_levels": (_c_int, [_vp]),
    "sam_model_num_points": (_c_int, [_vp, _c_int]),
    "sam_model_num_angles": (_c_int, [_vp, _c_int]),
    "sam_model_template_size": (_c_int, [_vp, _c_int, _i32p, _i32p]),
    "sam_model_rotated_points": (_c_int, [_vp, _c_int, _c_int, _i32p, _i32p, _f32p, _f32p]),
    "sam_model_points": (_c_int, [_vp, _c_int, _i32p, _i32p, _i32p, _i32p]),
    "sam_model_child_shift": (_c_int, [_vp, _c_int, _c_int, _i32p, _i32p]),
    "sam_detect": (_c_int, [_vp, _vp, _c_int, _c_int, _c_int, _c_int, ctypes.POINTER(DetectParams), _vp,
                            ctypes.POINTER(Pose), _c_int, ctypes.POINTER(_c_int)]),
    "sam_detect_batch": (_c_int, [_vp, _vp, _c_int, ctypes.c_size_t, _c_int, _c_int, _c_int, _c_int,
                                  ctypes.POINTER(DetectParams), _vp, ctypes.POINTER(Pose), _c_int,
                                  ctypes.POINTER(_c_int)]),
    "sam_pyramid_down": (_c_int, [_vp, _c_int, _c_int, _c_int, _vp, _c_int, _vp]),
    "sam_pyramid_levels": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp]),
    "sam_gradient": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _vp, _vp, _vp, _vp]),
    "sam_score_map": (_c_int, [_vp, _c_int, _vp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_float,
                               _c_int, _vp, _vp]),
    "sam_score_window_scratch_bytes": (ctypes.c_size_t, [ctypes.c_size_t]),
    "sam_score_window": (_c_int, [_vp, _c_int, _vp, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int, _c_int,
                                  _c_int, _c_int, _c_float, _c_int, _vp, _vp, ctypes.c_size_t, _vp, _vp]),
    "sam_set_score_kernel": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, _c_int]),
    "sam_get_score_kernel": (None, [_i32p, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "sam_take_device_error": (_c_int, []),
    "sam_selftest_wait_timeout": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_double)]),
    "sam_selftest_task_wait_timeout": (_c_int, [_c_int, ctypes.POINTER(ctypes.c_double)]),
    "sam_autotune": (_c_int, [_vp, _vp, _c_int, ctypes.c_size_t, _c_int, _c_int, _c_int, ctypes.POINTER(DetectParams),
                              _vp, _i32p, _f32p, _c_int, ctypes.POINTER(_c_int)]),
    "sam_model_tiling": (_c_int, [_vp, _c_int, _c_int, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "sam_candidates_scratch_bytes": (ctypes.c_size_t, [_c_int, _c_int, _c_int]),
    "sam_candidates": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_float, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "sam_candidates_scaled_scratch_bytes": (ctypes.c_size_t, [_c_int, _c_int, _c_int, _c_int]),
    "sam_candidates_scaled": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _c_float, _c_int, _vp, _vp, _vp, _vp,
                                       _vp]),
    "sam_candidates_noalloc": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_float, _c_int, _vp, _vp, _vp, _vp]),
    "sam_multi_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _i32p, _c_int, ctypes.c_void_p, _c_int,
                                  ctypes.POINTER(DetectParams), ctypes.POINTER(_vp)]),
    "sam_multi_free": (None, [_vp]),
    "sam_multi_image": (ctypes.c_void_p, [_vp, _c_int, ctypes.POINTER(_c_int)]),
    "sam_multi_set_image": (_c_int, [_vp, _c_int, _vp, _c_int, _c_int, _vp]),
    "sam_multi_run": (_c_int, [_vp, _vp, ctypes.POINTER(Pose), _c_int, ctypes.POINTER(_c_int)]),
    "sam_multi_set_tiling": (_c_int, [_vp, _c_int, _c_int, _c_int, _c_int, _c_int]),
    "sam_multi_autotune": (_c_int, [_vp, _vp, _i32p, _f32p, _c_int, ctypes.POINTER(_c_int)]),
    "sam_multi_stats": (_c_int, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_size_t)]),
    "sam_multi_pair_map": (_c_int, [_vp, _c_int, _vp, ctypes.c_size_t, ctypes.POINTER(_c_int),
                                    ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), ctypes.POINTER(_c_int), _vp]),
    "sam_score_bilinear": (_c_int, [_vp, _c_int, ctypes.POINTER(FieldRef), _c_int, _vp, _vp, _c_int, _vp, _vp, _vp,
                                    _vp]),
    "sam_score_bilinear_adjoint": (_c_int, [_vp, _c_int, ctypes.POINTER(FieldRef), _c_int, _vp, _vp, _c_int, _vp,
                                            _vp, _vp]),
    "sam_refine_poses": (_c_int, [_vp, _c_int, ctypes.POINTER(FieldRef), _c_int, _vp, _vp, _c_int, _c_int, _vp, _vp]),
    "sam_subpixel_poses": (_c_int, [_vp, ctypes.POINTER(FieldRef), _c_int, _vp, _vp, _c_int, _c_int, _vp, _vp]),
    "sam_response_maps_bytes": (ctypes.c_size_t, [_c_int, _c_int, _c_int]),
    "sam_score_map_quantized": (_c_int, [_vp, _c_int, _vp, _c_int, _c_int, _c_int, _c_int, _vp, ctypes.c_size_t,
                                         _vp, _vp]),
    "sam_profile_enable": (None, [_c_int]),
    "sam_set_graph_mode": (None, [_c_int]),
    "sam_profile_read": (_c_int, [_f32p, _i32p, _c_int]),
    "sam_kernel_launches": (ctypes.c_longlong, []),
    "sam_executed_pose_points": (ctypes.c_longlong, [_c_int]),
}

STAGES = ("pyramid", "gradient", "score_map", "candidates", "refine", "nms", "score_tiled")

_lib = None


class SamError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


def lib(build_if_missing: bool = True):
    """Load libsam.so (building it first if sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_str(s):
    return lib().sam_status_str(int(s)).decode()


def _check(s, where):
    if s != SAM_OK:
        raise SamError(s, where)


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def default_detect_params(**kw) -> DetectParams:
    p = DetectParams()
    lib().sam_default_detect_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


class Model:
    """A template model (sam_create_model): the template's edge points at every
    pyramid level (Sec. II edge extraction, hysteresis between `low` and
    `high`) and per level and angle index the Eq. (2) tables.  With
    scales=(scale_min, scale_step, n_scales) a scaled model
    (sam_create_model_scaled): tables per (scale, angle), Eq. (2) with
    A = s R(theta)."""

    def __init__(self, template: np.ndarray, low=30, high=60, levels=3, angle_step_deg=1.0, polarity=0,
                 scales=None):
        t = np.ascontiguousarray(template, dtype=np.uint8)
        if t.ndim != 2:
            raise ValueError("template must be a 2-D uint8 array")
        self.params = ModelParams(int(low), int(high), int(levels), float(angle_step_deg), int(polarity))
        h = ctypes.c_void_p()
        if scales is None:
            _check(lib().sam_create_model(t.ctypes.data_as(_vp), t.shape[1], t.shape[0], t.shape[1],
                                          ctypes.byref(self.params), ctypes.byref(h)), "sam_create_model")
        else:
            smin, sstep, ns = scales
            _check(lib().sam_create_model_scaled(t.ctypes.data_as(_vp), t.shape[1], t.shape[0], t.shape[1],
                                                 ctypes.byref(self.params), float(smin), float(sstep), int(ns),
                                                 ctypes.byref(h)), "sam_create_model_scaled")
        self._h = h
        self.levels = lib().sam_model_levels(h)

    def num_scales(self):
        return int(lib().sam_model_num_scales(self._h))

    def scale(self, j):
        return float(lib().sam_model_scale(self._h, int(j)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().sam_free_model(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_points(self, level):
        """n, the number of model points at `level` (Eq. (1)'s normaliser)."""
        return lib().sam_model_num_points(self._h, level)

    def num_angles(self, level):
        """Angle indices searched at `level` (360 / (angle_step * 2^level))."""
        return lib().sam_model_num_angles(self._h, level)

    def template_size(self, level):
        """(w, h) of the template at `level`."""
        w, h = ctypes.c_int32(), ctypes.c_int32()
        lib().sam_model_template_size(self._h, level, ctypes.byref(w), ctypes.byref(h))
        return w.value, h.value

    def rotated_points(self, level, k):
        """Eq. (2) table of (level, k): int32 offsets ox, oy and FP32 unit directions px, py."""
        n = self.num_points(level)
        ox, oy = np.empty(n, np.int32), np.empty(n, np.int32)
        px, py = np.empty(n, np.float32), np.empty(n, np.float32)
        _check(lib().sam_model_rotated_points(self._h, level, k, ox.ctypes.data_as(_i32p), oy.ctypes.data_as(_i32p),
                                              px.ctypes.data_as(_f32p), py.ctypes.data_as(_f32p)),
               "sam_model_rotated_points")
        return ox, oy, px, py

    def points(self, level):
        """The level's points: template coordinates tx, ty and integer Sobel gx, gy."""
        n = self.num_points(level)
        a = [np.empty(n, np.int32) for _ in range(4)]
        _check(lib().sam_model_points(self._h, level, *[x.ctypes.data_as(_i32p) for x in a]), "sam_model_points")
        return tuple(a)

    def child_shift(self, level, k_parent):
        """Coarse-to-fine shift: a level+1 pose (x, y, k_parent) maps to 2 (x, y) + shift."""
        sx, sy = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sam_model_child_shift(self._h, level, k_parent, ctypes.byref(sx), ctypes.byref(sy)),
               "sam_model_child_shift")
        return sx.value, sy.value


# sam_pose as a numpy record (the same 32 bytes), for reading whole result
# arrays at once
_POSE_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("theta_deg", "<f4"), ("score", "<f4"), ("angle_index", "<i4"),
                        ("level0_x", "<i4"), ("level0_y", "<i4"), ("scale_index", "<i4")])
assert _POSE_DTYPE.itemsize == ctypes.sizeof(Pose)


def _pose_lists(out, cap, counts) -> List[List[dict]]:
    """Pose dicts of consecutive result blocks of `cap` sam_pose each, the
    first counts[i] of block i."""
    rows = np.frombuffer(out, dtype=_POSE_DTYPE)
    res = []
    for i, n in enumerate(counts):
        res.append([dict(x=r[5], y=r[6], theta_deg=r[2], score=r[3], k=r[4], j=r[7])
                    for r in rows[i * cap:i * cap + n].tolist()])
    return res


def _poses(arr, n) -> List[dict]:
    return _pose_lists(arr, n, [n])[0]


def detect(model: Model, image, params: Optional[DetectParams] = None, stream=None, capacity=None):
    """sam_detect (Sec. II): detect the model in one image (numpy host array or
    torch CUDA uint8 tensor); a list of pose dicts (x, y, theta_deg, score, k) at
    level 0, best first."""
    params = params or default_detect_params()
    cap = capacity or params.max_detections
    out = (Pose * cap)()
    n = ctypes.c_int()
    if isinstance(image, np.ndarray):
        img = np.ascontiguousarray(image, dtype=np.uint8)
        ptr, on_dev, h, w, stride = img.ctypes.data_as(_vp), 0, img.shape[0], img.shape[1], img.shape[1]
        keep = img
    else:
        if not image.is_cuda or image.dtype.__str__() != "torch.uint8" or image.dim() != 2:
            raise ValueError("device images must be 2-D torch.uint8 CUDA tensors")
        if image.stride(1) != 1:
            raise ValueError("rows must be contiguous")
        ptr, on_dev, h, w, stride = _ptr(image), 1, image.shape[0], image.shape[1], image.stride(0)
        keep = image
    _check(lib().sam_detect(model.handle, ptr, w, h, stride, on_dev, ctypes.byref(params),
                            _stream(stream) if on_dev or _has_cuda() else None, out, cap, ctypes.byref(n)),
           "sam_detect")
    del keep
    return _poses(out, n.value)


def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def detect_batch(model: Model, images, params: Optional[DetectParams] = None, stream=None, capacity=None,
                 as_arrays=False):
    """sam_detect_batch (Sec. II, per image): detect in a (N, H, W) uint8 batch,
    a torch CUDA tensor or a host torch tensor / numpy array (copied by the
    library; pinned host memory makes the copy asynchronous); returns one pose
    list per image, or with as_arrays the library's results as they are: an
    (N, capacity) numpy record array of sam_pose (fields of Pose) and the
    (N,) int32 array of poses per image."""
    params = params or default_detect_params()
    cap = capacity or params.max_detections
    if isinstance(images, np.ndarray):
        keep = np.ascontiguousarray(images, dtype=np.uint8)
        N, H, W = keep.shape
        ptr, on_dev, strides = keep.ctypes.data_as(_vp), 0, (H * W, W)
    else:
        if images.dtype.__str__() != "torch.uint8" or images.dim() != 3:
            raise ValueError("images: a (N, H, W) uint8 tensor")
        N, H, W = images.shape
        if images.stride(2) != 1 or images.stride(1) < W:
            raise ValueError("rows must be contiguous")
        keep, ptr, on_dev, strides = images, _ptr(images), 1 if images.is_cuda else 0, (images.stride(0),
                                                                                          images.stride(1))
    out = (Pose * (cap * N))()
    nout = (ctypes.c_int * N)()
    _check(lib().sam_detect_batch(model.handle, ptr, N, strides[0], W, H, strides[1], on_dev, ctypes.byref(params),
                                  _stream(stream), out, cap, nout), "sam_detect_batch")
    del keep
    if as_arrays:
        return (np.frombuffer(out, dtype=_POSE_DTYPE).reshape(N, cap),
                np.frombuffer(nout, dtype=np.int32))
    return _pose_lists(out, cap, nout)


# ---- individual steps on torch CUDA tensors ----

def pyramid_down(src, dst, stream=None):
    """sam_pyramid_down (Sec. II image pyramid): dst = the 2x2 rounded mean of src
    (device uint8 tensors, 2-D, rows contiguous)."""
    h, w = src.shape
    _check(lib().sam_pyramid_down(_ptr(src), w, h, src.stride(0), _ptr(dst), dst.stride(0), _stream(stream)),
           "sam_pyramid_down")


def pyramid_levels(src, dsts, stream=None):
    """sam_pyramid_levels (Sec. II image pyramid): levels 1 .. len(dsts) of the
    device uint8 image src in one launch, level l into dsts[l - 1] (device
    uint8 tensors of at least floor(h / 2^l) x floor(w / 2^l), rows
    contiguous)."""
    h, w = src.shape
    n = len(dsts)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(d) for d in dsts])
    strides = (ctypes.c_int * n)(*[d.stride(0) for d in dsts])
    _check(lib().sam_pyramid_levels(_ptr(src), w, h, src.stride(0), n + 1, ptrs, strides, _stream(stream)),
           "sam_pyramid_levels")


def field_pitch(w, layout, precision=FP32):
    """Row pitch in pixels of a field of width w in the given layout (angle
    codes: 16-byte rows of 8 codes in the pairs layout)."""
    if precision == ANGLE16:
        return (w + 7) & ~7 if layout == LAYOUT_PAIRS else w
    return (w + 3) & ~3 if layout == LAYOUT_PAIRS else w


def angle_codes(img, low, stream=None, layout=None):
    """SAM_ANGLE16 field of a device uint8 image (sam_gradient): an (H, pitch)
    int16 CUDA tensor of 16-bit angle codes, pairs layout (pitch a multiple of
    8) unless `layout` says otherwise."""
    import torch
    h, w = img.shape
    layout = LAYOUT_PAIRS if layout is None else layout
    codes = torch.empty((h, field_pitch(w, layout, ANGLE16)), dtype=torch.int16, device=img.device)
    gradient(img, low, ANGLE16, codes, stream=stream, layout=layout)
    return codes


def gradient(img, low, precision, field, gx=None, gy=None, stream=None, layout=None):
    """sam_gradient (Sec. II edge extraction): Sobel gradients of a device uint8
    image, edges by the `low` threshold, unit field written to `field` in
    `precision` and `layout`; optional int16 gx, gy outputs."""
    h, w = img.shape
    layout = LAYOUT_PIXEL if layout is None else layout
    _check(lib().sam_gradient(_ptr(img), w, h, img.stride(0), int(low), int(precision), int(layout), _ptr(field),
                              _ptr(gx), _ptr(gy), _stream(stream)), "sam_gradient")


def score_map(model: Model, level, field, w, h, precision, out, step_x=1, step_y=1, nbhd=3, min_score=0.0,
              early=0, stream=None, layout=None):
    """sam_score_map: the exhaustive Eq. (1) score of every pose of the step grid
    at one level (points projected by Eq. (2)), written to out[k, y, x];
    with `early`, poses proved below min_score are -inf."""
    layout = LAYOUT_PIXEL if layout is None else layout
    _check(lib().sam_score_map(model.handle, int(level), _ptr(field), int(w), int(h), int(precision), int(layout),
                               int(step_x), int(step_y), int(nbhd), float(min_score), int(early), _ptr(out),
                               _stream(stream)), "sam_score_map")


def score_window_scratch_bytes(max_rescored):
    """Device bytes of score_window's FP32 rescoring list for up to max_rescored poses."""
    return int(lib().sam_score_window_scratch_bytes(int(max_rescored)))


def score_window(model: Model, level, field, w, h, precision, x0, y0, gw, gh, k0, nk, out, nbhd=3, min_score=0.0,
                 early=0, field32=None, scratch=None, stream=None):
    """Scores of the pose window [x0, x0+gw) x [y0, y0+gh) x angles [k0, k0+nk)
    into out (nk, gh, gw); field is the level's pairs-layout field."""
    nbytes = scratch.numel() * scratch.element_size() if scratch is not None else 0
    _check(lib().sam_score_window(model.handle, int(level), _ptr(field), int(w), int(h), int(precision), int(x0),
                                  int(y0), int(gw), int(gh), int(k0), int(nk), int(nbhd), float(min_score), int(early),
                                  _ptr(field32), _ptr(scratch), nbytes, _ptr(out), _stream(stream)),
           "sam_score_window")


def set_score_kernel(kernel=0, sx=2, sy=1, tg=9, warps=8, cols=6):
    """Select the exhaustive scorer: 0 automatic, 1 generic, 2 tiled (with its
    tiling; tg = 0 selects the chunked kernel; cols = pose columns per thread)."""
    _check(lib().sam_set_score_kernel(int(kernel), int(sx), int(sy), int(tg), int(warps), int(cols)),
           "sam_set_score_kernel")


def get_score_kernel():
    """The process-wide scorer selection (sam_get_score_kernel) as a dict."""
    v = [ctypes.c_int32() for _ in range(6)]
    lib().sam_get_score_kernel(*[ctypes.byref(x) for x in v])
    return dict(zip(("kernel", "sx", "sy", "tg", "warps", "cols"), (x.value for x in v)))


def take_device_error():
    """1 if a bounded wait of the scorers gave up since the last call (then cleared), else 0."""
    return int(lib().sam_take_device_error())


def selftest_wait_timeout(limit_us=2000):
    """Run the bounded-wait self-test; returns (status, milliseconds waited).
    The expected status is SAM_ERR_TIMEOUT."""
    ms = ctypes.c_double()
    s = int(lib().sam_selftest_wait_timeout(int(limit_us), ctypes.byref(ms)))
    return s, ms.value


def selftest_task_wait_timeout(limit_us=2000):
    """The persistent scorer's task wait on a task nothing publishes; returns
    (status, milliseconds waited).  The expected status is SAM_ERR_TIMEOUT."""
    ms = ctypes.c_double()
    s = int(lib().sam_selftest_task_wait_timeout(int(limit_us), ctypes.byref(ms)))
    return s, ms.value


def candidates_scratch_bytes(nth, gh, gw):
    """Device scratch bytes sam_candidates needs for an (nth, gh, gw) map."""
    return int(lib().sam_candidates_scratch_bytes(nth, gh, gw))


def candidates_scaled_scratch_bytes(n_scales, n_angles, gh, gw):
    """Device bytes of sam_candidates_scaled's scratch."""
    return int(lib().sam_candidates_scaled_scratch_bytes(int(n_scales), int(n_angles), int(gh), int(gw)))


def candidates_scaled(smap, min_score, K, out_kyx, out_s, count, scratch, stream=None):
    """sam_candidates_scaled: strict local maxima over (scale, angle circular,
    y, x) of a (n_scales, n_angles, gh, gw) score map; (plane, y, x) triples."""
    ns, na, gh, gw = smap.shape
    _check(lib().sam_candidates_scaled(_ptr(smap), ns, na, gh, gw, float(min_score), int(K), _ptr(out_kyx),
                                       _ptr(out_s), _ptr(count), _ptr(scratch), _stream(stream)),
           "sam_candidates_scaled")


def candidates(smap, min_score, K, out_kyx, out_s, count, scratch, stream=None):
    """sam_candidates: strict 3x3x3 local maxima (angle circular) of a score map
    at or above min_score, the best K (Sec. II returns the best pose; several
    instances read as local maxima)."""
    nth, gh, gw = smap.shape
    _check(lib().sam_candidates(_ptr(smap), nth, gh, gw, float(min_score), int(K), _ptr(out_kyx), _ptr(out_s),
                                _ptr(count), _ptr(scratch), _stream(stream)), "sam_candidates")


def set_graph_mode(on=True):
    """Replay the detection pipeline as a captured CUDA graph (default on)."""
    lib().sam_set_graph_mode(1 if on else 0)


def profile_enable(on=True):
    """Turn per-stage CUDA-event timing of sam_detect / sam_detect_batch on or off."""
    lib().sam_profile_enable(1 if on else 0)


def profile_read():
    """Per-stage device milliseconds and call counts since the last read."""
    n = len(STAGES)
    ms = (ctypes.c_float * n)()
    calls = (ctypes.c_int32 * n)()
    lib().sam_profile_read(ms, calls, n)
    return {STAGES[i]: (float(ms[i]), int(calls[i])) for i in range(n)}


def executed_pose_points(reset=False):
    """Pose-points the tiled scorers evaluated since the last reset (synchronises)."""
    v = int(lib().sam_executed_pose_points(1 if reset else 0))
    if v < 0:
        raise SamError(SAM_ERR_CUDA, "sam_executed_pose_points")
    return v


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(lib().sam_kernel_launches())


def candidates_noalloc(smap, min_score, K, out_kyx, out_s, count, stream=None):
    """sam_candidates using the library's fixed device scratch (no allocation,
    no scratch argument); for callers that cannot allocate device memory when
    they need candidates.  Calls that overlap on the GPU must be serialised."""
    nth, gh, gw = smap.shape
    _check(lib().sam_candidates_noalloc(_ptr(smap), nth, gh, gw, float(min_score), int(K), _ptr(out_kyx),
                                        _ptr(out_s), _ptr(count), _stream(stream)), "sam_candidates_noalloc")


def autotune(model: Model, images, params: Optional[DetectParams] = None, stream=None, max_out=512):
    """Time every tiling of the tiled scorer on a (N, H, W) uint8 CUDA batch and keep
    the fastest for `model`.  Returns a list of ((sx, sy, tg, warps), ms) sorted by time."""
    params = params or default_detect_params()
    N, H, W = images.shape
    cfg = (ctypes.c_int32 * (5 * max_out))()
    ms = (ctypes.c_float * max_out)()
    n = ctypes.c_int()
    _check(lib().sam_autotune(model.handle, _ptr(images), N, images.stride(0), W, H, images.stride(1),
                              ctypes.byref(params), _stream(stream), cfg, ms, max_out, ctypes.byref(n)),
           "sam_autotune")
    res = [(tuple(cfg[5 * i:5 * i + 5]), float(ms[i])) for i in range(n.value)]
    return sorted(res, key=lambda r: r[1])


def model_tiling(model: Model, precision=FP32, count=2):
    """(sx, sy, tg, warps, cols) the model's next calls with `precision` over
    `count` images use (count 1: the single-image class)."""
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().sam_model_tiling(model.handle, int(precision), int(count), *[ctypes.byref(x) for x in v]),
           "sam_model_tiling")
    return tuple(x.value for x in v)


class MultiPlan:
    """A batch of (image, model) pairs over images of different sizes, run as
    one captured CUDA graph with a persistent exhaustive scorer."""

    def __init__(self, models, image_sizes, pairs, params: Optional[DetectParams] = None):
        self.params = params or default_detect_params()
        self.models = list(models)   # keep the models alive
        n_m = len(self.models)
        mh = (_vp * n_m)(*[m.handle for m in self.models])
        sizes = (ctypes.c_int32 * (2 * len(image_sizes)))(*[v for wh in image_sizes for v in wh])
        pr = (ctypes.c_int * (2 * len(pairs)))(*[v for p in pairs for v in p])
        h = ctypes.c_void_p()
        _check(lib().sam_multi_create(mh, n_m, sizes, len(image_sizes), ctypes.cast(pr, ctypes.c_void_p),
                                      len(pairs), ctypes.byref(self.params), ctypes.byref(h)), "sam_multi_create")
        self._h = h
        self.image_sizes = list(image_sizes)
        self.n_pairs = len(pairs)

    def close(self):
        if getattr(self, "_h", None):
            lib().sam_multi_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_image(self, i, image, stream=None):
        """Copy image i (2-D uint8 numpy array or CUDA tensor) into the plan."""
        if isinstance(image, np.ndarray):
            img = np.ascontiguousarray(image, dtype=np.uint8)
            _check(lib().sam_multi_set_image(self._h, i, img.ctypes.data_as(_vp), img.shape[1], 0, _stream(stream)),
                   "sam_multi_set_image")
            import torch
            torch.cuda.current_stream().synchronize()
        else:
            _check(lib().sam_multi_set_image(self._h, i, _ptr(image), image.stride(0), 1, _stream(stream)),
                   "sam_multi_set_image")

    def run(self, stream=None, capacity=None):
        cap = capacity or self.params.max_detections
        out = (Pose * (cap * self.n_pairs))()
        nout = (ctypes.c_int * self.n_pairs)()
        _check(lib().sam_multi_run(self._h, _stream(stream), out, cap, nout), "sam_multi_run")
        return _pose_lists(out, cap, nout)

    def set_tiling(self, sx, sy, tg, warps, cols=6):
        _check(lib().sam_multi_set_tiling(self._h, sx, sy, tg, warps, cols), "sam_multi_set_tiling")

    def autotune(self, stream=None, max_out=256):
        cfg = (ctypes.c_int32 * (5 * max_out))()
        ms = (ctypes.c_float * max_out)()
        n = ctypes.c_int()
        _check(lib().sam_multi_autotune(self._h, _stream(stream), cfg, ms, max_out, ctypes.byref(n)),
               "sam_multi_autotune")
        res = [(tuple(cfg[5 * i:5 * i + 5]), float(ms[i])) for i in range(n.value)]
        return sorted(res, key=lambda r: r[1])

    def pair_map(self, pair, stream=None):
        """Pair `pair`'s top-level score map (sam_multi_pair_map) as a new
        (nth, gh, gw) float32 CUDA tensor, and the pyramid level it scores."""
        import torch
        nth, gh, gw, lvl = (ctypes.c_int() for _ in range(4))
        shape = lambda: (ctypes.byref(nth), ctypes.byref(gh), ctypes.byref(gw), ctypes.byref(lvl))  # noqa: E731
        _check(lib().sam_multi_pair_map(self._h, int(pair), None, 0, *shape(), _stream(stream)), "sam_multi_pair_map")
        out = torch.empty((nth.value, gh.value, gw.value), dtype=torch.float32, device="cuda")
        _check(lib().sam_multi_pair_map(self._h, int(pair), _ptr(out), out.numel(), *shape(), _stream(stream)),
               "sam_multi_pair_map")
        return out, lvl.value

    def stats(self):
        pp, gk, db = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t()
        _check(lib().sam_multi_stats(self._h, ctypes.byref(pp), ctypes.byref(gk), ctypes.byref(db)), "sam_multi_stats")
        return {"pose_points": pp.value, "graph_kernels": gk.value, "device_bytes": db.value}


# ---------------------------------------------------------------------------
# differentiable score on continuous poses
# ---------------------------------------------------------------------------

def unit_field(img, low, stream=None):
    """FP32 unit gradient field (H, W, 2) of a uint8 CUDA image, pixel layout."""
    import torch
    h, w = img.shape
    field = torch.empty((h, w, 2), dtype=torch.float32, device=img.device)
    gradient(img, low, FP32, field, stream=stream, layout=LAYOUT_PIXEL)
    return field


def _field_refs(fields):
    """ctypes array of FieldRef for a list of (H, W, 2) float32 CUDA tensors
    (row pitch may exceed W: a view with strides (2 P, 2, 1))."""
    import torch
    if len(fields) < 1 or len(fields) > MAX_BILINEAR_FIELDS:
        raise ValueError(f"between 1 and {MAX_BILINEAR_FIELDS} fields per call")
    refs = (FieldRef * len(fields))()
    for i, f in enumerate(fields):
        if f.dtype != torch.float32 or f.dim() != 3 or f.shape[2] != 2 or not f.is_cuda \
                or f.stride(2) != 1 or f.stride(1) != 2 or f.stride(0) % 2:
            raise ValueError("fields are (H, W, 2) float32 CUDA tensors with unit inner strides")
        refs[i] = FieldRef(f.data_ptr(), f.shape[1], f.shape[0], f.stride(0) // 2)
    return refs


def _poses_arg(poses):
    import torch
    if poses.dtype != torch.float32 or poses.dim() != 2 or poses.shape[1] != 3 or not poses.is_contiguous():
        raise ValueError("poses are a contiguous (B, 3) float32 CUDA tensor of (x, y, theta_deg)")
    return poses


def _pose_field_arg(pose_field, B):
    import torch
    if pose_field is None:
        return None
    if pose_field.dtype != torch.int32 or pose_field.numel() != B or not pose_field.is_contiguous():
        raise ValueError("pose_field is a contiguous int32 CUDA tensor with one entry per pose")
    return pose_field


def score_bilinear(model: Model, fields, poses, pose_field=None, level=0, grad=False, normal=False, stream=None):
    """Continuous-pose score M_c of each pose (B,); with grad=True also
    dM_c/d(x, y, theta_deg) (B, 3); with normal=True also the Gauss-Newton
    normal equations (B, 9): J^T J packed (xx, xy, xt, yy, yt, tt), J^T r."""
    import torch
    poses = _poses_arg(poses)
    B = poses.shape[0]
    pf = _pose_field_arg(pose_field, B)
    refs = _field_refs(fields)
    dev = poses.device
    score = torch.empty(B, dtype=torch.float32, device=dev)
    g = torch.empty((B, 3), dtype=torch.float32, device=dev) if grad else None
    nrm = torch.empty((B, 9), dtype=torch.float32, device=dev) if normal else None
    _check(lib().sam_score_bilinear(model.handle, int(level), refs, len(fields), _ptr(pf), _ptr(poses), B,
                                    _ptr(score), _ptr(g), _ptr(nrm), _stream(stream)), "sam_score_bilinear")
    out = [score] + ([g] if grad else []) + ([nrm] if normal else [])
    return out[0] if len(out) == 1 else tuple(out)


def score_bilinear_adjoint(model: Model, fields, poses, grad_score, pose_field=None, level=0, stream=None):
    """grad_score[b] * dM_c/d(x, y, theta_deg) at each pose, (B, 3)."""
    import torch
    poses = _poses_arg(poses)
    B = poses.shape[0]
    pf = _pose_field_arg(pose_field, B)
    refs = _field_refs(fields)
    gs = grad_score.to(torch.float32).contiguous()
    gp = torch.empty((B, 3), dtype=torch.float32, device=poses.device)
    _check(lib().sam_score_bilinear_adjoint(model.handle, int(level), refs, len(fields), _ptr(pf), _ptr(poses), B,
                                            _ptr(gs), _ptr(gp), _stream(stream)), "sam_score_bilinear_adjoint")
    return gp


def refine_poses(model: Model, fields, poses, pose_field=None, iterations=20, level=0, stream=None):
    """Damped Gauss-Newton refinement of (B, 3) poses in place (one launch);
    returns the final M_c per pose."""
    import torch
    poses = _poses_arg(poses)
    B = poses.shape[0]
    pf = _pose_field_arg(pose_field, B)
    refs = _field_refs(fields)
    score = torch.empty(B, dtype=torch.float32, device=poses.device)
    _check(lib().sam_refine_poses(model.handle, int(level), refs, len(fields), _ptr(pf), _ptr(poses), B,
                                  int(iterations), _ptr(score), _stream(stream)), "sam_refine_poses")
    return score


def response_maps_bytes(w, h, nbins):
    """Bytes of the response maps score_map_quantized needs for a w x h field."""
    return int(lib().sam_response_maps_bytes(int(w), int(h), int(nbins)))


def score_map_quantized(model: Model, level, field, nbins=16, neighbourhood=3, maps=None, stream=None):
    """Quantised-direction score map (num_angles, h, w) of an FP32 pixel-layout
    unit field (h, w, 2) CUDA tensor; `maps` optional scratch (uint8 tensor of
    response_maps_bytes) that holds the response maps afterwards."""
    import torch
    if field.dtype != torch.float32 or field.dim() != 3 or field.shape[2] != 2 or not field.is_contiguous():
        raise ValueError("field is a contiguous (h, w, 2) float32 CUDA tensor")
    h, w = field.shape[0], field.shape[1]
    nb = response_maps_bytes(w, h, nbins)
    if maps is None:
        maps = torch.empty(max(nb, 1), dtype=torch.uint8, device=field.device)
    out = torch.empty((model.num_angles(level), h, w), dtype=torch.float32, device=field.device)
    _check(lib().sam_score_map_quantized(model.handle, int(level), _ptr(field), w, h, int(nbins), int(neighbourhood),
                                         _ptr(maps), maps.numel() * maps.element_size(), _ptr(out), _stream(stream)),
           "sam_score_map_quantized")
    return out


def subpixel_poses(model: Model, fields, kyx, pose_field=None, neighbourhood=3, stream=None):
    """Sub-pixel / sub-angle poses of integer level-0 poses kyx (B, 3) int32 =
    (k, y, x) by the quadratic fit of their 3x3x3 score neighbourhood (one
    launch); returns a (B, 4) float32 tensor (x, y, theta_deg, M)."""
    import torch
    kyx = kyx.to(torch.int32).contiguous()
    if kyx.dim() != 2 or kyx.shape[1] != 3 or not kyx.is_cuda:
        raise ValueError("kyx is a (B, 3) CUDA tensor of (k, y, x)")
    B = kyx.shape[0]
    pf = _pose_field_arg(pose_field, B)
    refs = _field_refs(fields)
    out = torch.empty((B, 4), dtype=torch.float32, device=kyx.device)
    _check(lib().sam_subpixel_poses(model.handle, refs, len(fields), _ptr(pf), _ptr(kyx), B, int(neighbourhood),
                                    _ptr(out), _stream(stream)), "sam_subpixel_poses")
    return out


def _autograd_function():
    import torch

    class ScoreBilinear(torch.autograd.Function):
        """M_c(poses) with the library's adjoint kernel as backward.  The
        pose tensor is the only differentiable input."""

        @staticmethod
        def forward(ctx, poses, model, fields, pose_field, level):
            p = poses.detach().contiguous()
            ctx.save_for_backward(p)
            ctx.model, ctx.fields, ctx.pose_field, ctx.level = model, fields, pose_field, level
            return score_bilinear(model, fields, p, pose_field, level)

        @staticmethod
        def backward(ctx, grad_score):
            (p,) = ctx.saved_tensors
            gp = score_bilinear_adjoint(ctx.model, ctx.fields, p, grad_score.contiguous(), ctx.pose_field, ctx.level)
            return gp, None, None, None, None

    return ScoreBilinear


_SCORE_FN = None


def bilinear_score(poses, model: Model, fields, pose_field=None, level=0):
    """Differentiable M_c of (B, 3) poses (torch.autograd; backward runs the
    adjoint kernel)."""
    global _SCORE_FN
    if _SCORE_FN is None:
        _SCORE_FN = _autograd_function()
    return _SCORE_FN.apply(poses, model, list(fields), pose_field, int(level))

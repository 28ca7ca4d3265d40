"""GB300 (sm_103a) shape-based alignment detector after Le & Lin, arXiv 2112.05576.

The compute path is the CUDA library built from csrc/ (libsam.so, C ABI in
include/sam.h); this package is its thin Python binding.
"""

from .sam import (  # noqa: F401
    BF16,
    FP16,
    FP32,
    LAYOUT_PAIRS,
    LAYOUT_PIXEL,
    SIGNATURES,
    STAGES,
    DetectParams,
    FieldRef,
    MAX_BILINEAR_FIELDS,
    Model,
    ModelParams,
    MultiPlan,
    Pose,
    SamError,
    autotune,
    bilinear_score,
    candidates,
    candidates_noalloc,
    candidates_scratch_bytes,
    default_detect_params,
    detect,
    detect_batch,
    field_pitch,
    get_score_kernel,
    gradient,
    kernel_launches,
    lib,
    model_tiling,
    profile_enable,
    profile_read,
    pyramid_down,
    refine_poses,
    score_bilinear,
    score_bilinear_adjoint,
    score_map,
    set_score_kernel,
    status_str,
    take_device_error,
    unit_field,
)
from .build import build  # noqa: F401

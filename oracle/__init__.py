"""FP64 CPU oracle of the shape-based alignment detector (arXiv 2112.05576).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this package.  It
shares no code with the CUDA library; the arithmetic lives in
``sam_oracle.c`` (plain single-threaded C loops in FP64) and this module
only marshals numpy arrays and composes the steps in the paper's order:
edge extraction, pyramid, top-level exhaustive search, coarse-to-fine.
"""

from .oracle import (  # noqa: F401
    build,
    pyramid_down,
    pyramid,
    sobel,
    search_mask,
    hysteresis,
    unit_field,
    model_points,
    OracleModel,
    create_model,
    search_fields,
    rotate_points,
    score_pose,
    score_map,
    score_map_range,
    candidates,
    child_shift,
    refine_level,
    nms,
    detect,
    DetectParams,
    score_bilinear,
    bilinear_border_mask,
    refine_gn,
    subpixel_fit,
    neighbourhood27,
    climb27,
    subpixel_poses,
    quant_bin,
    score_map_quantized,
    response_maps,
    angle_codes,
    angle_field,
    search_angle_fields,
    project_affine,
    similarity,
    scale_grid,
    scaled_points,
    score_map_scaled,
    candidates_scaled,
    child_shift_scaled,
    refine_level_scaled,
    detect_scaled,
)

"""Seeded synthetic inputs shared by the tests, the oracle timing and the GPU benchmark.

This package only renders images (vector shapes, supersampling, noise,
illumination, occluders, clutter) and draws random poses.  It holds none of
the detector's arithmetic: no gradients, thresholds, pyramids or scores.
"""

from .scenes import (  # noqa: F401
    PartSpec,
    random_part,
    render_template,
    render_scene,
    tiny_case,
    config1_scene,
    config2_scene,
    config3_batch,
    config4_triples,
    config5_scene,
    paste_scene,
)

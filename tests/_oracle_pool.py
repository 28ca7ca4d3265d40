"""Oracle detections of many scenes in parallel worker processes.

Test infrastructure: the workers are spawned (never forked), so none of
them inherits a CUDA context from the test process.  Each worker builds the
oracle model from the template and runs oracle.detect on one scene; the
arithmetic is the oracle's alone.
"""

from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os


def _detect_one(job):
    import oracle
    tmpl, img, model_args, params = job
    om = oracle.create_model(tmpl, *model_args)
    return oracle.detect(om, img, oracle.DetectParams(**params))


def _score_map_one(job):
    import oracle
    tmpl, img, model_args, nbhd = job
    om = oracle.create_model(tmpl, *model_args)
    top = om.levels - 1
    field = oracle.search_fields(img, om.levels, om.low)[top]
    return oracle.score_map(field, om.points[top], om.ntheta(top), om.dtheta(top), nbhd=nbhd,
                            polarity=om.polarity)


def _detect_scaled_one(job):
    import oracle
    tmpl, img, model_args, scales, params = job
    om = oracle.create_model(tmpl, *model_args)
    return oracle.detect_scaled(om, img, oracle.DetectParams(**params), scales)


def _run(fn, jobs, workers=None):
    workers = workers or max(1, min(len(jobs), os.cpu_count() or 1, 16))
    if workers == 1 or len(jobs) == 1:
        return [fn(j) for j in jobs]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, jobs))


def detect_many(jobs, workers=None):
    """jobs: (template, scene, (low, high, levels, angle_step_deg[, polarity]), DetectParams kwargs) tuples;
    returns oracle.detect's list for each, in order."""
    return _run(_detect_one, jobs, workers)


def top_maps(jobs, workers=None):
    """jobs: (template, scene, model args, neighbourhood) tuples; returns the FP64 top-level score map of each."""
    return _run(_score_map_one, jobs, workers)


def detect_scaled_many(jobs, workers=None):
    """jobs: (template, scene, model args, scale grid, DetectParams kwargs) tuples; oracle.detect_scaled of each."""
    return _run(_detect_scaled_one, jobs, workers)

#!/usr/bin/env python3
"""Benchmark of the shape-based alignment detector on GB300.

Workload: the paper-shaped single detection at 1280x1024 -- a 200x200
texture-less part (about 1500 edge points at level 0), 1-4 instances per
scene with occlusion, an illumination ramp, clutter and noise; 4 pyramid
levels, 1 degree angle step at level 0 (8 degrees, 45 angles at the top),
neighbourhood 3, min_score 0.6.  One step = detection of one batch of
`--batch` such scenes resident in HBM (all pipeline stages: pyramid,
gradients, top-level exhaustive search, candidates, refinement to level 0,
NMS, result readback).

Metric: pose-point evals/s = (top-level poses x model points at the top
level) per second, summed over the batch (refinement work is not counted).

Arms: the default arm runs the CUDA library; --impl reference times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import tempfile
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

LEVELS, STEP, LOW, HIGH, MIN_SCORE = 4, 1.0, 30, 60, 0.6
W, H, SIDE = 1280, 1024, 200
METRIC = "pose-point evals/s (1280x1024 detection, top-level exhaustive)"
UNIT = "pose-point/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _scenes(n, seed0, spec=None):
    tm, imgs, truth = None, [], []
    for i in range(n):
        t, sc, gt, spec = synth.config2_scene(seed=seed0 + i, W=W, H=H, side=SIDE, spec=spec)
        tm = t if tm is None else tm
        imgs.append(sc)
        truth.append(gt)
    return tm, imgs, truth, spec


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        # raw samples (the summary goes into the JSON line); BENCH_CLOCKS_DIR
        # keeps them elsewhere
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"sam_bench_clocks_gpu{gpu}_{os.getpid()}.csv")

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for line in f if line.endswith("\n"))
        except OSError:
            return 0

    def _wait_lines(self, n, limit_s):
        t0 = time.perf_counter()
        while self._lines() < n and time.perf_counter() - t0 < limit_s:
            time.sleep(0.005)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            # the sampler is running before the timed region starts
            self._wait_lines(1, 5.0)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            # and takes one more sample after it (a region shorter than the
            # sampling interval still gets the samples on both sides)
            self._wait_lines(self._lines() + 1, 1.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def top_pose_points(model, batch):
    top = LEVELS - 1
    tw, th = W >> top, H >> top
    return batch * model.num_angles(top) * tw * th * model.num_points(top)


# ---------------------------------------------------------------------------
# roofline of the exhaustive scoring kernel
# ---------------------------------------------------------------------------
# The tiled FP32 kernel is bound by shared-memory bandwidth.  Each thread
# scores an 8 x 6 block of translations for one angle; for every model
# point it reads the (8 + 2) x (6 + 2) pixels under the block's 3 x 3
# windows from the staged FP32 field, 8 bytes per pixel: 640 bytes for 48
# pose-points, i.e. 13.33 algorithmic shared-memory bytes per pose-point.
# (16-bit fields: 4 bytes per pixel, half that.)  The chunked kernel uses
# the same block; the tiled kernel's 8 x 10 block needs 10 x 12 pixels per
# 80 poses, 12 bytes per pose-point (the figure quoted is the 8 x 6 one, so
# the fraction is conservative for it).
# Peak: 128 bytes/clk/SM x SMs x maximum SM clock.  Achieved counts the
# pose-points the kernel evaluated (the library's device counter: poses
# inside the map x points processed before early termination), so work that
# early termination skips is not credited; the nominal-count figure and the
# launch without early termination are reported beside it.
SMEM_B_PER_PP = 640.0 / 48.0
SMEM_B_PER_CLK_SM = 128.0
# Second bound, of the method itself with full reuse of the per-pixel dot
# products across the 3x3 window: the separable 3x3 maximum costs 4
# comparisons per pose-point on the ALU pipe, 128/clk/SM with the 3-input max.
CMP_PER_PP = 4
CMP_PER_CLK_SM = 128.0


# With early termination the detection path scores the top level with one
# persistent kernel (score_fused_kernel) doing two kinds of work: the
# edge-presence bound of every pose (a bit-sliced count of the points whose
# 3x3 window holds an edge pixel; poses that cannot reach min_score are
# written -inf) and the dot products of the surviving poses, a lane scoring a
# 2 x TC slice.  Per model point the slice reads (2 + 2) x (TC + 2) staged
# pixels for 2 x TC poses: 19.2 bytes per pose-point at TC 10, 21.3 at TC 6
# (FP32 fields; 16-bit fields half).
DRAIN_ROWS = 2


def slice_bytes_per_pp(cols, precision):
    px = 8.0 if precision == "fp32" else 4.0
    return (DRAIN_ROWS + 2) * (cols + 2) * px / (DRAIN_ROWS * cols)


# The bound's algorithmic work, bit-parallel over 32 poses per word: per
# model point and pose word one funnel-shift extraction of the dilated edge
# bitmap and a 3-operation carry-save full adder, 4 logical operations per 32
# pose-points; against 64 32-bit logical operations per clock per SM
# (nominal integer throughput, not measured).
BOUND_OPS_PER_PP = 4.0 / 32.0
LOGIC_OPS_PER_CLK_SM = 64.0

# DRAM bytes (read + write) of one score_fused_kernel launch of this
# workload, from ncu captures at the tilings below (sx, sy, tg, warps, cols);
# reported only when the headline runs one of them, and to be re-taken
# whenever the kernel changes.  The headline prefers a captured tiling when
# the autotuner timed it within PREFER_PROFILED of the fastest.
NCU_FUSED_TRAFFIC = {(2, 1, 12, 8, 6): 2969088 + 6661376, (1, 1, 23, 8, 6): 2972928 + 6584576}
PREFER_PROFILED = 1.02


def dense_roofline(pp_per_launch, ms_per_launch, sm_count, sm_mhz_peak, traffic=None):
    """Shared-memory roofline of the dense tiled scorer (every pose scored,
    8 x 6 block, 13.33 B per pose-point) and its 3 x 3 maximum on the ALU."""
    sec = ms_per_launch * 1e-3
    achieved = pp_per_launch * SMEM_B_PER_PP / sec / 1e12
    peak = SMEM_B_PER_CLK_SM * sm_count * sm_mhz_peak * 1e6 / 1e12
    alu_ach = pp_per_launch * CMP_PER_PP / sec / 1e12
    alu_peak = CMP_PER_CLK_SM * sm_count * sm_mhz_peak * 1e6 / 1e12
    return {"bound": "smem", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "kernel": "score_tiled_kernel (dense: every pose of the top level scored)",
            "alu": {"achieved": round(alu_ach, 3), "peak": round(alu_peak, 3), "unit": "Tcmp/s",
                    "frac": round(alu_ach / alu_peak, 4)}}


# ---------------------------------------------------------------------------
# CPU oracle timing
# ---------------------------------------------------------------------------

def oracle_sample(budget_s=20.0, seed=9000):
    import oracle
    tm, imgs, _, _ = _scenes(1, seed)
    om = oracle.create_model(tm, LOW, HIGH, LEVELS, STEP)
    top = LEVELS - 1
    pp_one = om.ntheta(top) * (W >> top) * (H >> top) * len(om.points[top][0])
    params = oracle.DetectParams(min_score=MIN_SCORE, nbhd=3)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.detect(om, imgs[0], params)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s * 0.5 or n >= 8:
            break
    return pp_one * n / el, el, n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    tm, imgs, _, _ = _scenes(1, 9000)
    om = oracle.create_model(tm, LOW, HIGH, LEVELS, STEP)
    top = LEVELS - 1
    nth = om.ntheta(top)
    tw, th = W >> top, H >> top
    n_top = len(om.points[top][0])
    field = oracle.search_fields(imgs[0], LEVELS, LOW)[top]
    # A step scores a slice of m top-level angles over every translation (the
    # oracle's exhaustive search is >95 % of its detection time); m is sized
    # so warm-up + timed steps take about two minutes.
    t0 = time.perf_counter()
    oracle.score_map_range(field, om.points[top], 0, 1, om.dtheta(top), nbhd=3)
    t_angle = time.perf_counter() - t0
    m = int(max(1, min(nth, 120.0 / max(1e-6, (args.steps + args.warmup) * t_angle))))
    for i in range(args.warmup):
        oracle.score_map_range(field, om.points[top], (i * m) % (nth - m + 1), m, om.dtheta(top), nbhd=3)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.score_map_range(field, om.points[top], (i * m) % (nth - m + 1), m, om.dtheta(top), nbhd=3)
    el = time.perf_counter() - t0
    val = m * tw * th * n_top * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "config2: 1280x1024 scene, 200x200 part, 4 levels, dtheta 1 deg, nbhd 3, "
                               "min_score 0.6", "batch": 1,
                   "sample": f"top-level exhaustive scoring of {m} of {nth} angles per step"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x {m} top-level angles x {tw}x{th} translations x "
                                   f"{n_top} points, FP64 oracle, single thread"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# batched uneven form (config 3 shape)
# ---------------------------------------------------------------------------

def levels_for_side(side):
    """Pyramid levels of a template: 3 up to 96 px, else 4 (360 one-degree
    angles halve exactly three times: 360, 180, 90, 45)."""
    return 3 if side <= 96 else 4


def run_batched(args, sam, torch, dev, stream):
    tmpls, images, pairs, _ = synth.config3_batch(n_images=args.multi)
    models = [sam.Model(t, LOW, HIGH, levels_for_side(t.shape[0]), STEP) for t in tmpls]
    sizes = [(im.shape[1], im.shape[0]) for im in images]
    out = {"images": len(images), "pairs": len(pairs), "templates": [t.shape[0] for t in tmpls],
           "workload": "config3: 64 images of 640x480..2592x1944, 8 templates 64..400 px, 2 per image"}
    for name, code in (("fp32", 0), ("bf16", 1), ("fp16", 2)):
        params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                           precision=code, early_termination=1)
        plan = sam.MultiPlan(models, sizes, pairs, params)
        for i, im in enumerate(images):
            plan.set_image(i, torch.from_numpy(im).to(dev))
        tuning = plan.autotune()
        for _ in range(3):
            res = plan.run()
        st = plan.stats()
        n = max(5, min(20, args.steps))
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            res = plan.run()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / n
        out[name] = {"value": st["pose_points"] / (ms * 1e-3), "unit": UNIT, "ms_per_batch": round(ms, 3),
                     "ms_per_pair": round(ms / len(pairs), 4), "pose_points_per_batch": st["pose_points"],
                     "graph_kernels": st["graph_kernels"], "runs": n,
                     "tiling": tuning[0][0] if tuning else None,
                     "detections": int(sum(len(r) for r in res))}
        plan.close()
    # the same pairs through the single-image path, one detect call per pair
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                       precision=0, early_termination=1)
    dimgs = [torch.from_numpy(im).to(dev) for im in images]
    for i, m in pairs[:8]:
        sam.detect(models[m], dimgs[i], params)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i, m in pairs:
        sam.detect(models[m], dimgs[i], params)
    torch.cuda.synchronize(dev)
    ms = (time.perf_counter() - t0) * 1e3
    out["sequential_fp32"] = {"ms_per_batch": round(ms, 3), "ms_per_pair": round(ms / len(pairs), 4),
                              "value": out["fp32"]["pose_points_per_batch"] / (ms * 1e-3), "unit": UNIT,
                              "what": "one detect call per pair (single-image path), host-timed"}
    return out


# ---------------------------------------------------------------------------
# differentiable form (config 4 shape)
# ---------------------------------------------------------------------------

def _event_ms(torch, dev, stream, fn, reps):
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        fn(i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / reps


def run_differentiable(args, sam, torch, dev, stream, with_oracle):
    n_tr = args.refine
    tmpl, imgs, triples = synth.config4_triples(n=n_tr)
    model = sam.Model(tmpl, LOW, HIGH, LEVELS, STEP)
    fields = [sam.unit_field(torch.from_numpy(im).to(dev), LOW) for im in imgs]
    init = torch.tensor([t[2] for t in triples], dtype=torch.float32, device=dev)
    gt = np.array([t[1] for t in triples], dtype=np.float64)
    pf = torch.tensor([t[0] for t in triples], dtype=torch.int32, device=dev)
    npts = model.num_points(0)
    reps = 20
    out = {"workload": f"config4: {n_tr} (scene, pose) pairs, 4 scenes 1280x1024, 200x200 part "
                       f"({npts} level-0 points), start +-1.5 px / +-1.5 deg from truth",
           "poses": n_tr, "points": npts}
    # forward alone, and forward + backward through the autograd Function
    for _ in range(3):
        sam.score_bilinear(model, fields, init, pf)
    ms_f = _event_ms(torch, dev, stream, lambda i: sam.score_bilinear(model, fields, init, pf), reps)
    ones = torch.ones(n_tr, device=dev)

    def fb(i):
        p = init.clone().requires_grad_(True)
        sam.bilinear_score(p, model, fields, pf).backward(ones)

    for _ in range(3):
        fb(0)
    ms_fb = _event_ms(torch, dev, stream, fb, reps)
    out["forward"] = {"ms": round(ms_f, 4), "point_evals_per_s": n_tr * npts / (ms_f * 1e-3)}
    out["forward_backward"] = {"ms": round(ms_fb, 4), "point_evals_per_s": 2 * n_tr * npts / (ms_fb * 1e-3),
                               "kernels": 2}
    # 20 Gauss-Newton iterations, one launch (21 evaluations per pose)
    copies = [init.clone() for _ in range(reps + 3)]
    for i in range(3):
        sam.refine_poses(model, fields, copies[reps + i], pf, iterations=20)
    ms_r = _event_ms(torch, dev, stream, lambda i: sam.refine_poses(model, fields, copies[i], pf, iterations=20), reps)
    got = copies[0].cpu().numpy().astype(np.float64)
    err = np.abs(got - gt)
    ok = (err[:, 0] < 0.05) & (err[:, 1] < 0.05) & (err[:, 2] < 0.05)
    out["refine"] = {"iterations": 20, "ms": round(ms_r, 4), "us_per_pose": round(ms_r * 1e3 / n_tr, 3),
                     "point_evals_per_s": 21 * n_tr * npts / (ms_r * 1e-3),
                     "within_0.05px_0.05deg": round(float(ok.mean()), 4),
                     "median_err": [round(float(v), 4) for v in np.median(err, 0)],
                     "p95_err": [round(float(v), 4) for v in np.percentile(err, 95, axis=0)],
                     "start_within": round(float(((np.abs(init.cpu().numpy() - gt) < 0.05).all(1)).mean()), 4)}
    if with_oracle:
        import oracle
        om = oracle.create_model(tmpl, LOW, HIGH, LEVELS, STEP)
        ofs = [oracle.search_fields(im, 1, LOW)[0] for im in imgs]
        t0 = time.perf_counter()
        k = 0
        while k < n_tr and (k < 8 or time.perf_counter() - t0 < args.cpu_budget / 4):
            oracle.refine_gn(ofs[triples[k][0]], om.points[0], triples[k][2], iterations=20)
            k += 1
        el = time.perf_counter() - t0
        out["refine"]["cpu_baseline"] = {"us_per_pose": round(el * 1e6 / k, 1), "cores": 1, "kind": "oracle",
                                         "sample": f"{k} poses, 20 iterations, FP64 oracle, one thread"}
    return out


# ---------------------------------------------------------------------------
# large exhaustive stress slice (config 5 shape)
# ---------------------------------------------------------------------------

def run_stress(args, sam, torch, dev, stream):
    tmpl, img, poses = synth.config5_scene()
    H5, W5 = img.shape
    step5 = 0.5
    model = sam.Model(tmpl, LOW, HIGH, 1, step5)
    n = model.num_points(0)
    nth = model.num_angles(0)
    dimg = torch.from_numpy(img).to(dev)
    fields = {}
    for prec, dt in ((0, torch.float32), (1, torch.bfloat16)):
        wp = sam.field_pitch(W5, sam.LAYOUT_PAIRS)
        f = torch.empty((H5, wp, 2), dtype=dt, device=dev)
        sam.gradient(dimg, LOW, prec, f, layout=sam.LAYOUT_PAIRS)
        fields[prec] = f
    field32 = torch.empty((H5, W5, 2), dtype=torch.float32, device=dev)
    sam.gradient(dimg, LOW, 0, field32, layout=sam.LAYOUT_PIXEL)
    x, y, th = poses[0]
    k = int(round(th / step5)) % nth
    slices = {"angles8_full_image": (0, 0, W5, H5, min(max(0, k - 4), nth - 8), 8),
              "all_angles_512x512": (int(x) - 256, int(y) - 256, 512, 512, 0, nth)}
    scratch = torch.empty(sam.score_window_scratch_bytes(1 << 22), dtype=torch.uint8, device=dev)
    out = {"workload": f"config5: {W5}x{H5} image, 512x512 part ({n} points), dtheta {step5} deg ({nth} angles), "
                       f"level 0 only, step 1 px, nbhd 3, min_score 0.6",
           "points": n, "full_search_pose_points": nth * W5 * H5 * n}
    peaks, _ = _peaks()
    smem_peak = SMEM_B_PER_CLK_SM * torch.cuda.get_device_properties(dev).multi_processor_count * \
        float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    reps = 3
    for name, win in slices.items():
        x0, y0, gw, gh, k0, nk = win
        omap = torch.empty((nk, gh, gw), dtype=torch.float32, device=dev)
        pp = nk * gw * gh * n
        res = {"window": list(win), "pose_points": pp}
        for label, prec, early, f32 in (("fp32", 0, 1, None), ("fp32_no_early_termination", 0, 0, None),
                                        ("bf16_rescored", 1, 1, field32)):
            def call(i, prec=prec, early=early, f32=f32):
                sam.score_window(model, 0, fields[prec], W5, H5, prec, x0, y0, gw, gh, k0, nk, omap, nbhd=3,
                                 min_score=0.6, early=early, field32=f32, scratch=scratch if f32 is not None else None)
            call(0)
            sam.executed_pose_points(reset=True)
            ms = _event_ms(torch, dev, stream, call, reps)
            ex = sam.executed_pose_points(reset=True) / reps
            res[label] = {"ms": round(ms, 3), "value": pp / (ms * 1e-3), "unit": UNIT,
                          "edge_presence_bound": bool(early),
                          "executed_pose_points": int(ex),
                          "smem_frac": round(ex * SMEM_B_PER_PP * (1.0 if prec == 0 else 0.5) / (ms * 1e-3) / 1e12
                                             / smem_peak, 4),
                          "best": round(float(omap.max()), 5)}
        out[name] = res
    rate = out["angles8_full_image"]["fp32"]["value"]
    out["extrapolated_full_search_s"] = {
        "fp32": round(out["full_search_pose_points"] / rate, 1),
        "bf16_rescored": round(out["full_search_pose_points"] / out["angles8_full_image"]["bf16_rescored"]["value"], 1)}
    return out


# ---------------------------------------------------------------------------
# sub-pixel / sub-angle final pose
# ---------------------------------------------------------------------------

def run_subpixel(args, sam, torch, dev, stream, model, spec, n_scenes=8):
    """The quadratic fit of the 3x3x3 Eq. (1) neighbourhood (neighbourhoods 3
    and 1) and the Gauss-Newton refinement of the continuous score, on config-2
    scenes whose instances sit at sub-pixel positions (U(-1/2, 1/2) px) and on a
    0.5 degree angle grid, against the rendered truth."""
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16)
    rows, kyx, owner, fields = [], [], [], []
    for i in range(n_scenes):
        _, sc, gts, _ = synth.config2_scene(seed=9100 + i, W=W, H=H, side=SIDE, spec=spec, subpixel=True)
        img = torch.from_numpy(sc).to(dev)
        fields.append(sam.unit_field(img, LOW))
        for d in sam.detect(model, img, params):
            gx, gy, gth = min(gts, key=lambda t: (t[0] - d["x"]) ** 2 + (t[1] - d["y"]) ** 2)
            if (gx - d["x"]) ** 2 + (gy - d["y"]) ** 2 > 9:
                continue   # a detection of no instance
            kyx.append((d["k"], d["y"], d["x"]))
            owner.append(i)
            rows.append((gx, gy, gth))
    if not kyx:
        return None
    k_t = torch.tensor(kyx, dtype=torch.int32, device=dev)
    o_t = torch.tensor(owner, dtype=torch.int32, device=dev)
    for _ in range(3):
        sam.subpixel_poses(model, fields, k_t, o_t)
    ms = _event_ms(torch, dev, stream, lambda i: sam.subpixel_poses(model, fields, k_t, o_t), 20)
    f3 = sam.subpixel_poses(model, fields, k_t, o_t, neighbourhood=3).cpu().numpy()
    f1 = sam.subpixel_poses(model, fields, k_t, o_t, neighbourhood=1).cpu().numpy()
    gn = torch.tensor([(float(x), float(y), float(k) * STEP) for k, y, x in kyx], dtype=torch.float32, device=dev)
    sam.refine_poses(model, fields, gn, o_t, iterations=20)
    gn = gn.cpu().numpy()
    ang = lambda a, b: abs(((a - b) + 180.0) % 360.0 - 180.0)  # noqa: E731
    err = {"integer": [], "fit_nbhd3": [], "fit_nbhd1": [], "gauss_newton": []}
    for (k, y, x), (gx, gy, gth), a, b, g in zip(kyx, rows, f3, f1, gn):
        err["integer"].append((math.hypot(x - gx, y - gy), ang(k * STEP, gth)))
        err["fit_nbhd3"].append((math.hypot(a[0] - gx, a[1] - gy), ang(float(a[2]), gth)))
        err["fit_nbhd1"].append((math.hypot(b[0] - gx, b[1] - gy), ang(float(b[2]), gth)))
        err["gauss_newton"].append((math.hypot(g[0] - gx, g[1] - gy), ang(float(g[2]) % 360.0, gth)))
    out = {"what": "quadratic fit of the 3x3x3 Eq. (1) neighbourhood (sam_subpixel_poses, one launch) and 20 "
                   "Gauss-Newton steps of the bilinear score, from the integer detections of config-2 scenes with "
                   "instances at sub-pixel positions; errors against the rendered truth",
           "scenes": n_scenes, "poses": len(kyx), "ms": round(ms, 4), "us_per_pose": round(1e3 * ms / len(kyx), 3)}
    for name, e in err.items():
        a = np.array(e)
        out[name] = {"mean_pos_err_px": round(float(a[:, 0].mean()), 4),
                     "mean_angle_err_deg": round(float(a[:, 1].mean()), 4)}
    return out


# ---------------------------------------------------------------------------
# field storage forms on the exhaustive top-level map
# ---------------------------------------------------------------------------

def run_storage_forms(args, sam, torch, dev, stream, model, batch):
    """The top level (160 x 128, 45 angles) of each config-2 scene of one batch
    scored exhaustively with sam_score_map from an FP32 pairs field, a BF16
    pairs field and an angle-code field (SAM_ANGLE16), every pose scored and
    with early termination (the persistent scorer); field bytes, time per map
    and the largest score difference from the FP32 map."""
    top = LEVELS - 1
    imgs = []
    for i in range(batch.shape[0]):
        lvl = batch[i].contiguous()
        for _ in range(top):
            nxt = torch.empty((lvl.shape[0] // 2, lvl.shape[1] // 2), dtype=torch.uint8, device=dev)
            sam.pyramid_down(lvl, nxt)
            lvl = nxt
        imgs.append(lvl)
    th, tw = imgs[0].shape
    nth, n = model.num_angles(top), model.num_points(top)
    fields = {}
    for name, prec, dt in (("fp32", sam.FP32, torch.float32), ("bf16", sam.BF16, torch.bfloat16),
                           ("angle16", sam.ANGLE16, torch.int16)):
        wp = sam.field_pitch(tw, sam.LAYOUT_PAIRS, prec)
        fl = []
        for im in imgs:
            f = torch.empty((th, wp) if prec == sam.ANGLE16 else (th, wp, 2), dtype=dt, device=dev)
            sam.gradient(im, LOW, prec, f, layout=sam.LAYOUT_PAIRS)
            fl.append(f)
        fields[name] = (prec, fl, fl[0].numel() * fl[0].element_size())
    maps = [torch.empty((nth, th, tw), dtype=torch.float32, device=dev) for _ in imgs]
    out = {"what": f"sam_score_map of the {tw}x{th} top level, {nth} angles, {n} points, of {len(imgs)} config-2 "
                   "scenes, one call per scene, each form with the tiling the autotuner picks for it (one image "
                   "per call; angle codes take the FP32 tiling); error = max |M - M_fp32| over every pose (early "
                   "termination off)",
           "pose_points_per_map": nth * th * tw * n}
    ref = None
    one = batch[:1].contiguous()
    for early in (0, 1):
        key = "early_termination" if early else "every_pose"
        out[key] = {}
        # the scorer's tiling for one image per call, per stored form and mode
        for prec in (sam.FP32, sam.BF16):
            sam.autotune(model, one, sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, precision=prec,
                                                               early_termination=early))
        for name, (prec, fl, fbytes) in fields.items():
            def call(i, prec=prec, fl=fl, early=early):
                j = i % len(fl)
                sam.score_map(model, top, fl[j], tw, th, prec, maps[j], 1, 1, 3, MIN_SCORE, early,
                              layout=sam.LAYOUT_PAIRS)
            for i in range(len(imgs)):
                call(i)
            ms = _event_ms(torch, dev, stream, call, 4 * len(imgs))
            res = {"ms_per_map": round(ms, 4), "value": out["pose_points_per_map"] / (ms * 1e-3), "unit": UNIT,
                   "field_bytes": int(fbytes),
                   "tiling": list(sam.model_tiling(model, sam.FP32 if prec == sam.ANGLE16 else prec, 1))}
            if not early:
                cur = torch.stack(maps).cpu().numpy()
                if name == "fp32":
                    ref = cur
                res["max_abs_err_vs_fp32"] = float(np.max(np.abs(cur - ref)))
            out[key][name] = res
    out["angle16_bound"] = round(2 * math.sin(math.pi / 65536), 7)
    return out


# ---------------------------------------------------------------------------
# scaled poses (Eq. (2) with A = s R(theta))
# ---------------------------------------------------------------------------

SCALE_GRID = (0.9, 0.1, 3)     # 0.9, 1.0, 1.1


def run_scaled(args, sam, torch, dev, stream, tm, spec, n_scenes=8):
    """Detection over scales x angles x translations (a scaled model,
    sam_create_model_scaled) on config-2 scenes whose instances are drawn at
    the grid's scales, next to the rigid model on the same scenes: time per
    batch (device-resident, graph replay), nominal pose-points, and the
    instances found at their scale."""
    grid = [SCALE_GRID[0] + j * SCALE_GRID[1] for j in range(SCALE_GRID[2])]
    imgs, truth = [], []
    for i in range(n_scenes):
        _, sc, gts, _ = synth.config2_scene(seed=9300 + i, W=W, H=H, side=SIDE, spec=spec, scales=grid)
        imgs.append(sc)
        truth.append(gts)
    batch = torch.from_numpy(np.stack(imgs)).to(dev)
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16)
    out = {"what": f"sam_detect_batch of {n_scenes} config-2 scenes with instances at scales {grid}; scaled model "
                   f"(scales {grid}) vs the rigid model, autotuned tilings, early termination",
           "scales": grid}
    for name, model in (("scaled", sam.Model(tm, LOW, HIGH, LEVELS, STEP, scales=SCALE_GRID)),
                        ("rigid", sam.Model(tm, LOW, HIGH, LEVELS, STEP))):
        sam.autotune(model, batch, params)
        for _ in range(3):
            res = sam.detect_batch(model, batch, params)
        ms = _event_ms(torch, dev, stream, lambda i: sam.detect_batch(model, batch, params), 10)
        top = LEVELS - 1
        pp = n_scenes * model.num_scales() * model.num_angles(top) * (W >> top) * (H >> top) * model.num_points(top)
        found, right_scale = 0, 0
        for dets, gts in zip(res, truth):
            for gx, gy, gth, gs in gts:
                near = [d for d in dets if (d["x"] - gx) ** 2 + (d["y"] - gy) ** 2 <= 9]
                if near:
                    found += 1
                    right_scale += int(abs(model.scale(near[0]["j"]) - gs) < 1e-9)
        out[name] = {"ms_per_batch": round(ms, 4), "ms_per_detection": round(ms / n_scenes, 5),
                     "value": pp / (ms * 1e-3), "unit": UNIT, "pose_points_per_batch": pp,
                     "instances": int(sum(len(t) for t in truth)), "found": found, "found_at_their_scale": right_scale}
    return out


# ---------------------------------------------------------------------------
# HBM-bound kernels (a) gradient and (b) pyramid on images larger than L2
# ---------------------------------------------------------------------------
# Algorithmic bytes: the gradient kernel reads each 8-bit pixel once and
# writes its unit-field pixel once (8 B FP32 pair, 4 B 16-bit pair; pairs
# layout, row pitch rounded up to 4 pixels); the pyramid kernel reads the
# 2 x 2 block of 8-bit pixels under each output pixel and writes it (4 + 1 B).
# DRAM bytes (read + write) per launch, from an ncu capture of
# `bench.py --only hbm --steps 1` (mean over the captured launches), keyed by
# kernel, field form and image size.  Writes that are still in L2 when a
# launch ends are not counted, so a field that fits L2 shows less write
# traffic than it has algorithmic bytes.
NCU_HBM_TRAFFIC = {
    ("gradient_kernel", "fp32", 4096, 3072): 48_818_000,
    ("gradient_kernel", "bf16", 4096, 3072): 12_607_000,
    ("gradient_kernel", "fp32_pixel", 4096, 3072): 48_655_000,
    ("pyramid_down_kernel", 4096, 3072): 12_589_000,
    ("gradient_kernel", "fp32", 8192, 6144): 387_774_000,
    ("gradient_kernel", "bf16", 8192, 6144): 187_279_000,
    ("gradient_kernel", "fp32_pixel", 8192, 6144): 387_699_000,
    ("pyramid_down_kernel", 8192, 6144): 50_340_000,
}


def _hbm_images(torch, dev, n, W_, H_):
    """n distinct W_ x H_ uint8 device images cut from shifted config-5 scenes."""
    _, img5, _ = synth.config5_scene()
    rng = np.random.default_rng(77)
    reps_y, reps_x = -(-H_ // img5.shape[0]), -(-W_ // img5.shape[1])
    big = np.tile(img5, (reps_y, reps_x))
    out = []
    for _ in range(n):
        sh = np.roll(big, (int(rng.integers(0, big.shape[0])), int(rng.integers(0, big.shape[1]))), axis=(0, 1))
        out.append(torch.from_numpy(np.ascontiguousarray(sh[:H_, :W_])).to(dev))
    return out


def run_hbm(args, sam, torch, dev, stream):
    peaks, kind = _peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    out = {"peak_gbs": peak, "peak_source": f"{kind} hbm_gbs (STREAM-style copy)",
           "what": "per-launch CUDA-event time of back-to-back launches over distinct buffers "
                   "(working set several times the 129 MB L2)"}
    for label, (W_, H_, n, reps) in (("config5_4096x3072", (4096, 3072, 8, 40)),
                                     ("mosaic_8192x6144", (8192, 6144, 3, 12))):
        reps = min(reps, max(1, args.steps))
        srcs = _hbm_images(torch, dev, n, W_, H_)
        res = {}
        for name, prec, layout, dt, bpx in (("fp32", sam.FP32, sam.LAYOUT_PAIRS, torch.float32, 8),
                                            ("bf16", sam.BF16, sam.LAYOUT_PAIRS, torch.bfloat16, 4),
                                            ("fp32_pixel", sam.FP32, sam.LAYOUT_PIXEL, torch.float32, 8),
                                            ("angle16", sam.ANGLE16, sam.LAYOUT_PAIRS, torch.int16, 2)):
            wp = sam.field_pitch(W_, layout, prec)
            shape = (H_, wp) if prec == sam.ANGLE16 else (H_, wp, 2)
            dsts = [torch.empty(shape, dtype=dt, device=dev) for _ in range(n)]
            call = (lambda i, dsts=dsts, prec=prec, layout=layout:
                    sam.gradient(srcs[i % n], LOW, prec, dsts[i % n], layout=layout))
            for i in range(3):
                call(i)
            ms = _event_ms(torch, dev, stream, call, reps)
            alg = W_ * H_ + H_ * wp * bpx
            gbs = alg / (ms * 1e-3) / 1e9
            res["gradient_" + name] = {
                "bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
                "traffic": NCU_HBM_TRAFFIC.get(("gradient_kernel", name, W_, H_)), "algorithmic_bytes": alg,
                "us_per_launch": round(ms * 1e3, 2)}
            del dsts
        dsts = [torch.empty((H_ // 2, W_ // 2), dtype=torch.uint8, device=dev) for _ in range(n)]
        call = lambda i: sam.pyramid_down(srcs[i % n], dsts[i % n])  # noqa: E731
        for i in range(3):
            call(i)
        ms = _event_ms(torch, dev, stream, call, reps * 4)
        alg = 5 * (W_ // 2) * (H_ // 2)
        gbs = alg / (ms * 1e-3) / 1e9
        res["pyramid"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                          "frac": round(gbs / peak, 4), "traffic": NCU_HBM_TRAFFIC.get(("pyramid_down_kernel", W_, H_)),
                          "algorithmic_bytes": alg, "us_per_launch": round(ms * 1e3, 2)}
        del dsts
        # the detection pipeline's form: levels 1-3 in one launch (level 0
        # read once, the later levels from shared memory)
        lv = [[torch.empty((H_ >> l, W_ >> l), dtype=torch.uint8, device=dev) for l in (1, 2, 3)] for _ in range(n)]
        call = lambda i: sam.pyramid_levels(srcs[i % n], lv[i % n])  # noqa: E731
        for i in range(3):
            call(i)
        ms = _event_ms(torch, dev, stream, call, reps * 4)
        alg = W_ * H_ + sum((W_ >> l) * (H_ >> l) for l in (1, 2, 3))
        gbs = alg / (ms * 1e-3) / 1e9
        res["pyramid_levels"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                                 "frac": round(gbs / peak, 4), "traffic": None, "algorithmic_bytes": alg,
                                 "us_per_launch": round(ms * 1e3, 2)}
        out[label] = res
        del srcs, lv
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    import paper_2112_05576_gb300 as sam
    from paper_2112_05576_gb300 import shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sam.lib()
    B = args.batch
    pools = max(2, args.pools)
    tm, imgs, truth, spec = _scenes(B, 3000 + 7919 * rank)
    # further batches: circular shifts of the same scenes (distinct buffers,
    # so no batch is still in L2 when it is scored again)
    rng = np.random.default_rng(11 + rank)
    for _ in range(pools - 1):
        for i in range(B):
            imgs.append(np.roll(imgs[i], (int(rng.integers(0, H)), int(rng.integers(0, W))), axis=(0, 1)))
    model = sam.Model(tm, LOW, HIGH, LEVELS, STEP)
    params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                       precision={"fp32": 0, "bf16": 1, "fp16": 2}[args.precision],
                                       early_termination=1 if args.early else 0)
    host = np.stack(imgs).reshape(pools, B, H, W)
    batches = [torch.from_numpy(host[i]).to(dev) for i in range(pools)]
    pinned = torch.from_numpy(host).pin_memory()
    stream = torch.cuda.current_stream(dev)

    # the project's autotuner picks the scorer's tiling on this workload (setup,
    # outside every timed region)
    if args.tiling:
        sam.set_score_kernel(2, *(int(v) for v in args.tiling.split(",")))
    tuning = sam.autotune(model, batches[0], params) if (args.autotune and not args.tiling) else []
    head_tiling = tuple(sam.model_tiling(model, params.precision, B))
    profiled = [t for t, t_ms in tuning if tuple(t) in NCU_FUSED_TRAFFIC and t_ms <= tuning[0][1] * PREFER_PROFILED]
    if profiled:
        head_tiling = tuple(profiled[0])
        sam.set_score_kernel(2, *head_tiling)

    def step(i, as_arrays=False):
        return sam.detect_batch(model, batches[i % pools], params, as_arrays=as_arrays)

    # ---- device-resident timed region (the library's default graph mode) ----
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    launches0 = sam.kernel_launches()
    sam.executed_pose_points(reset=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(args.steps):
            res = step(i, as_arrays=True)   # poses in host memory, as the library returns them
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    launches = sam.kernel_launches() - launches0
    exec_pp = sam.executed_pose_points(reset=True) / max(1, args.steps)
    ms = shard.max_over_ranks(ev0.elapsed_time(ev1), device=dev)
    # stage times: the same K steps again with the library's stage events on
    # (which run the pipeline's launches directly, outside graph mode)
    sam.profile_enable(True)
    sam.profile_read()
    for i in range(args.steps):
        step(i)
    prof = sam.profile_read()
    sam.profile_enable(False)
    pp_step = top_pose_points(model, B)
    value = shard.whole_job_rate(pp_step, args.steps, world, ms)

    # ---- end to end through the public API with host buffers: one library
    # call per step takes the pinned host batch (its host-to-device copy is
    # inside the call, on the stream) and returns the poses in host memory ----
    h2d = B * H * W
    d2h = B * (params.max_detections * 32 + 4)
    for i in range(2):
        sam.detect_batch(model, pinned[i % pools], params)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        sam.detect_batch(model, pinned[i % pools], params, as_arrays=True)   # host images in, host poses out
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = shard.max_over_ranks(e0.elapsed_time(e1), device=dev)
    e2e_value = shard.whole_job_rate(pp_step, args.steps, world, e2e_ms)
    if profiled:
        sam.set_score_kernel(0)

    # ---- sub-pixel / sub-angle poses (scenes with off-grid instances) ----
    subpixel = None
    if rank == 0 and args.extras:
        subpixel = run_subpixel(args, sam, torch, dev, stream, model, spec)

    # ---- quantised-direction form (response maps) on one top level ----
    quantized = None
    if rank == 0 and args.extras:
        lvl = batches[0][0].contiguous()
        for _ in range(LEVELS - 1):
            hh, ww = lvl.shape
            nxt = torch.empty((hh // 2, ww // 2), dtype=torch.uint8, device=dev)
            sam.pyramid_down(lvl, nxt)
            lvl = nxt
        th_, tw_ = lvl.shape
        top_l = LEVELS - 1
        qfield = sam.unit_field(lvl, LOW)
        pfield = torch.zeros((th_, sam.field_pitch(tw_, sam.LAYOUT_PAIRS), 2), dtype=torch.float32, device=dev)
        sam.gradient(lvl, LOW, sam.FP32, pfield, layout=sam.LAYOUT_PAIRS)
        exact = torch.empty((model.num_angles(top_l), th_, tw_), dtype=torch.float32, device=dev)
        quantized = {"what": "one 160x128 top level, all 45 angles, every pose scored: response maps + gather-add "
                             "(sam_score_map_quantized) against the exact Eq. (1) map (sam_score_map, no early "
                             "termination)", "pose_points": int(exact.numel() * model.num_points(top_l))}
        for _ in range(3):
            sam.score_map(model, top_l, pfield, tw_, th_, sam.FP32, exact, 1, 1, 3, 0.0, 0, layout=sam.LAYOUT_PAIRS)
        ms_exact = _event_ms(torch, dev, stream, lambda i: sam.score_map(model, top_l, pfield, tw_, th_, sam.FP32,
                                                                         exact, 1, 1, 3, 0.0, 0,
                                                                         layout=sam.LAYOUT_PAIRS), 20)
        quantized["exact_ms"] = round(ms_exact, 4)
        ex = exact.cpu().numpy()
        for nb in (16, 32):
            qmaps = torch.empty(sam.response_maps_bytes(tw_, th_, nb), dtype=torch.uint8, device=dev)
            for _ in range(3):
                q = sam.score_map_quantized(model, top_l, qfield, nb, 3, maps=qmaps)
            ms_q = _event_ms(torch, dev, stream,
                             lambda i: sam.score_map_quantized(model, top_l, qfield, nb, 3, maps=qmaps), 20)
            err = np.abs(q.cpu().numpy() - ex)
            quantized[f"bins{nb}"] = {"ms": round(ms_q, 4), "max_abs_err": round(float(err.max()), 5),
                                      "mean_abs_err": round(float(err.mean()), 6),
                                      "bound": round(2 * math.sin(2 * math.pi / nb / 4), 5),
                                      "same_argmax": bool(int(np.argmax(q.cpu().numpy())) == int(np.argmax(ex)))}

    # ---- single-image latency (one detection, device-resident) ----
    one = batches[0][0].contiguous()
    # the scorer's tiling for one image per call is tuned on its own (setup)
    if args.autotune and not args.tiling:
        sam.autotune(model, one[None], params)
    for _ in range(3):
        sam.detect(model, one, params)
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    n_single = 50
    for _ in range(n_single):
        sam.detect(model, one, params)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    single_ms = s0.elapsed_time(s1) / n_single

    # ---- the 16-bit stored forms on the same batches (own tiling, FP32 rescoring) ----
    forms = {}
    if args.precision == "fp32" and args.forms:
        ref_dets = {i: step(i) for i in range(pools)}
        for name, code in (("fp16", 2), ("bf16", 1)):
            fp = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                           precision=code, early_termination=1 if args.early else 0)
            if args.autotune and not args.tiling:
                sam.autotune(model, batches[0], fp)
            same = all([(d["x"], d["y"], d["k"]) for d in a] == [(d["x"], d["y"], d["k"]) for d in b]
                       for i in range(pools)
                       for a, b in zip(sam.detect_batch(model, batches[i], fp), ref_dets[i]))
            n_form = max(10, min(50, args.steps))
            for i in range(3):
                sam.detect_batch(model, batches[i % pools], fp)
            torch.cuda.synchronize(dev)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for i in range(n_form):
                sam.detect_batch(model, batches[i % pools], fp, as_arrays=True)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            fms = f0.elapsed_time(f1) / n_form
            sam.profile_enable(True)
            sam.profile_read()
            for i in range(n_form):
                sam.detect_batch(model, batches[i % pools], fp)
            pf = sam.profile_read()
            sam.profile_enable(False)
            forms[name] = {"value": top_pose_points(model, B) / (fms * 1e-3), "ms_per_step": round(fms, 4),
                           "ms_per_detection": round(fms / B, 5),
                           "score_map_ms": round(pf["score_map"][0] / max(1, pf["score_map"][1]), 4),
                           "candidates_ms": round(pf["candidates"][0] / max(1, pf["candidates"][1]), 4),
                           "same_detections_as_fp32": bool(same), "steps": n_form,
                           "tiling": dict(zip(("sx", "sy", "tg", "warps", "cols"), sam.model_tiling(model, code, B)))}

    # ---- the batched uneven form: many image sizes and templates, one graph ----
    batched = run_batched(args, sam, torch, dev, stream) if (args.multi > 0 and rank == 0) else None

    # ---- the large exhaustive stress slice (chunked scorer) ----
    stress = run_stress(args, sam, torch, dev, stream) if (args.stress and rank == 0) else None

    # ---- scaled poses: the search over scales x angles x translations ----
    scaled = run_scaled(args, sam, torch, dev, stream, tm, spec) if (args.scaled and rank == 0) else None

    # ---- field storage forms (FP32 / BF16 pairs / angle codes) on one top-level map ----
    storage = run_storage_forms(args, sam, torch, dev, stream, model, batches[0]) if (rank == 0 and args.extras) \
        else None

    # ---- kernels (a) gradient and (b) pyramid against HBM ----
    hbm = run_hbm(args, sam, torch, dev, stream) if (args.hbm and rank == 0) else None

    # ---- the differentiable form: continuous-pose score, adjoint, refinement ----
    differentiable = (run_differentiable(args, sam, torch, dev, stream, world == 1 and not args.no_cpu)
                      if (args.refine > 0 and rank == 0) else None)

    # ---- the scorer with every pose fully evaluated (no early termination) ----
    full_params = sam.default_detect_params(min_score=MIN_SCORE, neighbourhood=3, top_k=64, max_detections=16,
                                            precision=params.precision, early_termination=0)
    for i in range(2):
        step_full = sam.detect_batch(model, batches[i % pools], full_params)
    sam.profile_enable(True)
    sam.profile_read()
    n_full = max(5, min(20, args.steps))
    for i in range(n_full):
        sam.detect_batch(model, batches[i % pools], full_params)
    prof_full = sam.profile_read()
    sam.profile_enable(False)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peaks, peak_kind = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = props.multi_processor_count
    score_ms, score_calls = prof["score_map"]
    tiling = head_tiling
    tiled_ms, tiled_calls = prof.get("score_tiled", (0.0, 0))
    smem_peak = SMEM_B_PER_CLK_SM * nsm * sm_mhz * 1e6 / 1e12
    if args.early and tiled_calls:
        # the persistent scorer: its dot products against the shared-memory
        # roofline, its bound against the logic-op one, and their sum
        k_ms = tiled_ms / tiled_calls
        bpp = slice_bytes_per_pp(tiling[4], args.precision)
        ach = exec_pp * bpp / (k_ms * 1e-3) / 1e12
        ops_peak = LOGIC_OPS_PER_CLK_SM * nsm * sm_mhz * 1e6 / 1e12
        ops_ach = pp_step * BOUND_OPS_PER_PP / (k_ms * 1e-3) / 1e12
        rl = {"bound": "smem", "achieved": round(ach, 3), "peak": round(smem_peak, 3), "unit": "TB/s",
              "frac": round(ach / smem_peak, 4),
              "traffic": args.traffic if args.traffic is not None else (
                  NCU_FUSED_TRAFFIC.get(tiling) if params.precision == 0 else None),
              "kernel": "score_fused_kernel (persistent: edge-presence bound of every pose, then the surviving "
                        "2-row slices)",
              "ms_per_launch": round(k_ms, 4),
              "peak_source": (f"{peak_kind} sm_max_mhz x {nsm} SMs x 128 shared-memory bytes/clk; "
                              f"{bpp:.2f} algorithmic bytes per executed pose-point (2 x {tiling[4]} slice)"),
              "alu": {"what": "the bound: 4 logical ops per 32 pose-points, all poses", "achieved": round(ops_ach, 3),
                      "peak": round(ops_peak, 3), "unit": "Tops/s", "frac": round(ops_ach / ops_peak, 4),
                      "peak_source": "nominal 64 logical ops/clk/SM x SMs x sm_max_mhz"},
              "combined_frac": round(ach / smem_peak + ops_ach / ops_peak, 4),
              "combined_what": "(dot-product time at the shared-memory peak + bound time at the logic-op peak) "
                               "/ kernel time",
              "score_map_ms_per_step": round(score_ms / max(1, score_calls), 4)}
    else:
        rl = dense_roofline(exec_pp, score_ms / max(1, score_calls), nsm, sm_mhz, traffic=args.traffic)
        rl["peak_source"] = (f"{peak_kind} sm_max_mhz x {nsm} SMs x 128 shared-memory "
                             f"bytes/clk; 13.33 algorithmic bytes per pose-point (8x6 translation block)")
        rl["ms_per_launch"] = round(score_ms / max(1, score_calls), 4)
    clocks = clk.summary()
    if clocks.get("sm_mhz"):
        rl["frac_at_observed_clock"] = round(rl["frac"] * sm_mhz / clocks["sm_mhz"], 4)
    fms, fcalls = prof_full["score_map"]
    rl_full = dense_roofline(pp_step, fms / max(1, fcalls), props.multi_processor_count,
                       float(peaks.get("sm_max_mhz", 2070.0)))
    rl["no_early_termination"] = {"ms_per_launch": round(fms / max(1, fcalls), 4), "achieved": rl_full["achieved"],
                                  "frac": rl_full["frac"], "bound": "smem",
                                  "what": "score_tiled_kernel, every pose fully scored, 13.33 B per pose-point"}
    rl_nom = dense_roofline(pp_step, score_ms / max(1, score_calls), props.multi_processor_count,
                      float(peaks.get("sm_max_mhz", 2070.0)))
    rl["executed_pose_points_per_launch"] = int(exec_pp)
    rl["nominal_pose_points_per_launch"] = int(pp_step)
    rl["nominal"] = {"achieved": rl_nom["achieved"], "frac": rl_nom["frac"],
                     "what": "nominal pose-points (early termination not subtracted) x 13.33 B / score-map time"}
    if hbm:
        # kernels (a) and (b) on the config-5 image, FP32 pairs field (the scored layout)
        c5 = hbm["config5_4096x3072"]
        rl["gradient_kernel"] = dict(c5["gradient_fp32"], image="4096x3072 -> FP32 pairs field")
        rl["pyramid_down_kernel"] = dict(c5["pyramid"], image="4096x3072 -> 2048x1536")
    rl["tiling"] = dict(zip(("sx", "sy", "tg", "warps", "cols"), head_tiling))
    rl["tiling"]["autotuned"] = bool(tuning)
    rl["tiling"]["profiled_preferred"] = bool(profiled)
    if tuning:
        rl["tiling"]["candidates"] = len(tuning)
        rl["tiling"]["best_ms"] = round(tuning[0][1], 4)
        rl["tiling"]["worst_ms"] = round(tuning[-1][1], 4)
    cpu = None
    if world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        v, el, n = oracle_sample(args.cpu_budget)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} full config-2 detection(s) of one 1280x1024 scene, FP64 oracle, "
                         f"single thread, {el:.1f} s"}
    stages = {k: {"ms_per_step": round(v[0] / max(1, args.steps), 4), "calls": v[1]} for k, v in prof.items()}
    ndet = [int(c) for c in res[1]]   # poses per image of the last timed step
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.precision if args.precision != "fp32" else "f32",
        "data": "synthetic",
        "config": {"workload": "config2: 1280x1024 scenes, 200x200 part (~1500 edge pts), 4 levels, "
                               "dtheta 1 deg (45 top angles), nbhd 3, min_score 0.6",
                   "batch": B, "early_termination": bool(args.early), "precision": args.precision,
                   "l2": f"inputs larger than L2: {pools} rotating batches, per-step working set "
                         f"~{B * (H * W * 11 // 1048576)} MB"},
        "ms_per_detection": ms / args.steps / B,
        "single_image_ms": single_ms,
        "single_image_value": top_pose_points(model, 1) / (single_ms * 1e-3),
        "executed": {"pose_points_per_step": int(exec_pp), "value": exec_pp * args.steps / (ms * 1e-3),
                     "unit": "executed pose-point/s",
                     "what": "pose-points the scorer actually evaluated (device counter) per second of the timed "
                             "steps; the headline counts the exhaustive-equivalent (nominal) pose-points"},
        "single_image_tiling": dict(zip(("sx", "sy", "tg", "warps", "cols"), sam.model_tiling(model, params.precision, 1))),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps,
                "what": "sam_detect_batch with the batch in pinned host memory (img_on_device = 0): the copy in "
                        "and the pose readback are inside the library call"},
        "gpu_launches": int(launches),
        "stages": stages,
        "stages_note": "per-stage device times from a second pass of the same steps with stage events on (direct launches); the timed steps replay the captured pipeline graph",
        "roofline": rl,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "detections_per_image": ndet[:8],
        "forms": forms,
        "batched": batched,
        "differentiable": differentiable,
        "subpixel": subpixel,
        "quantized": quantized,
        "stress": stress,
        "storage_forms": storage,
        "scaled": scaled,
        "hbm": hbm,
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_section(args):
    import torch

    import paper_2112_05576_gb300 as sam
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sam.lib()
    stream = torch.cuda.current_stream(dev)
    res = {"hbm": run_hbm, "stress": run_stress}[args.only](args, sam, torch, dev, stream)
    print(json.dumps({"section": args.only, "result": res}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--pools", type=int, default=4)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--early", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--forms", type=int, default=1, help="also time the FP16/BF16 stored forms")
    ap.add_argument("--multi", type=int, default=64, help="images of the batched uneven form (0: skip)")
    ap.add_argument("--refine", type=int, default=4096, help="poses of the differentiable form (0: skip)")
    ap.add_argument("--stress", type=int, default=1, help="time the config-5 stress slices (0: skip)")
    ap.add_argument("--hbm", type=int, default=1, help="time the gradient and pyramid kernels against HBM (0: skip)")
    ap.add_argument("--scaled", type=int, default=1, help="time the scaled-pose detection (0: skip)")
    ap.add_argument("--tiling", default="", help="force the tiled scorer's sx,sy,tg,warps[,cols] (no autotuning)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per score launch, if measured")
    ap.add_argument("--extras", type=int, default=1,
                    help="time the sub-pixel, quantised and storage-form sections (0: skip)")
    ap.add_argument("--only", default="", choices=["", "hbm", "stress"],
                    help="run one section alone and print its JSON (for profiling; not a bench line)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_section(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())

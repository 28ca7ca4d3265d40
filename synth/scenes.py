"""Vector-rendered synthetic templates and search scenes (seeded, numpy only).

A *part* is a union of filled primitives (polygons, circles, rings, slots)
minus hole primitives, defined in continuous template coordinates.  Pixel
(col, row) of an image has its centre at the continuous point (col, row).
Every image is rendered with 4x4 supersampling: the 16 sample points of a
pixel sit at offsets {-3/8, -1/8, 1/8, 3/8} from its centre in x and y, the
pixel value is floor(mean + 1/2) of the sample intensities.

An instance of a template of size W x H placed at pose (u_x, u_y, theta) maps
template point T to scene point q = R(theta) (T - c) + u with
c = (floor(W/2), floor(H/2)) and R the rotation of the plane in image
coordinates (x right, y down).  Scenes are rendered by mapping every scene
sample back, T = R(theta)^-1 (q - u) + c, and evaluating the part there, so
an instance is drawn at its pose rather than raster-rotated.  For theta a
multiple of 90 degrees and integer u the sample grid maps onto itself, so a
pasted instance is an exact permutation of the template's pixels.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_SUB = (np.arange(4, dtype=np.float64) + 0.5) / 4.0 - 0.5  # supersample offsets


# ----------------------------------------------------------------------------
# primitives
# ----------------------------------------------------------------------------

def _in_polygon(x, y, verts):
    """Even-odd point-in-polygon test for arrays of points."""
    inside = np.zeros(x.shape, dtype=bool)
    n = len(verts)
    for i in range(n):
        x0, y0 = verts[i]
        x1, y1 = verts[(i + 1) % n]
        if y0 == y1:
            continue
        cond = (y0 > y) != (y1 > y)
        xc = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
        inside ^= cond & (x < xc)
    return inside


def _in_prim(x, y, prim):
    kind = prim[0]
    if kind == "poly":
        return _in_polygon(x, y, prim[1])
    if kind == "circle":
        _, cx, cy, r = prim
        return (x - cx) ** 2 + (y - cy) ** 2 < r * r
    if kind == "ring":
        _, cx, cy, r0, r1 = prim
        d2 = (x - cx) ** 2 + (y - cy) ** 2
        return (d2 >= r0 * r0) & (d2 < r1 * r1)
    if kind == "slot":
        _, ax, ay, bx, by, r = prim
        vx, vy = bx - ax, by - ay
        ll = vx * vx + vy * vy
        t = np.clip(((x - ax) * vx + (y - ay) * vy) / ll, 0.0, 1.0)
        dx = x - (ax + t * vx)
        dy = y - (ay + t * vy)
        return dx * dx + dy * dy < r * r
    if kind == "rect":
        _, x0, y0, x1, y1 = prim
        return (x >= x0) & (x < x1) & (y >= y0) & (y < y1)
    raise ValueError(kind)


@dataclass
class PartSpec:
    """A texture-less part: filled primitives minus holes, in template coords."""

    width: int
    height: int
    fill: list = field(default_factory=list)
    holes: list = field(default_factory=list)
    part_level: float = 200.0
    background: float = 60.0

    def inside(self, x, y):
        m = np.zeros(x.shape, dtype=bool)
        for p in self.fill:
            m |= _in_prim(x, y, p)
        for p in self.holes:
            m &= ~_in_prim(x, y, p)
        return m

    def on_template(self, x, y):
        """True where the continuous point lies on the template's pixel grid."""
        return (x >= -0.5) & (x < self.width - 0.5) & (y >= -0.5) & (y < self.height - 0.5)


def _star_polygon(rng, cx, cy, rmin, rmax, nv):
    ang = np.sort(rng.uniform(0, 2 * math.pi, nv))
    # keep vertices angularly spread so the polygon is not degenerate
    ang = np.linspace(0, 2 * math.pi, nv, endpoint=False) + rng.uniform(-0.25, 0.25, nv) * (2 * math.pi / nv)
    rad = rng.uniform(rmin, rmax, nv)
    return [(cx + r * math.cos(a), cy + r * math.sin(a)) for a, r in zip(ang, rad)]


def random_part(rng, side, kind="tiny", margin=3.0):
    """A random part on a side x side template.

    kind="tiny":  one random filled polygon (5-8 vertices) plus one ring.
    kind="part":  an outer polygon body with circular holes and slots, sized
                  so a 200 x 200 template yields roughly 1500 edge pixels.
    Edges stay at least `margin` pixels inside the template border.
    """
    s = float(side)
    c = (side // 2, side // 2)
    spec = PartSpec(width=side, height=side)
    if kind == "tiny":
        nv = int(rng.integers(5, 9))
        rmax = s / 2 - margin
        poly = _star_polygon(rng, c[0], c[1], 0.45 * rmax, rmax, nv)
        spec.fill.append(("poly", poly))
        rr = rng.uniform(0.12, 0.2) * s
        ring_c = (c[0] + rng.uniform(-0.1, 0.1) * s, c[1] + rng.uniform(-0.1, 0.1) * s)
        # the ring is a dark band inside the polygon (hole) so it adds edges
        spec.holes.append(("ring", ring_c[0], ring_c[1], rr, rr + max(1.5, 0.05 * s)))
    elif kind == "part":
        nv = int(rng.integers(7, 11))
        rmax = s / 2 - margin
        body = _star_polygon(rng, c[0], c[1], 0.72 * rmax, rmax, nv)
        spec.fill.append(("poly", body))
        nh = int(rng.integers(2, 4))
        for _ in range(nh):
            r = rng.uniform(0.05, 0.09) * s
            a = rng.uniform(0, 2 * math.pi)
            d = rng.uniform(0.1, 0.3) * s
            spec.holes.append(("circle", c[0] + d * math.cos(a), c[1] + d * math.sin(a), r))
        ns = int(rng.integers(1, 3))
        for _ in range(ns):
            a = rng.uniform(0, 2 * math.pi)
            d = rng.uniform(0.05, 0.25) * s
            px, py = c[0] + d * math.cos(a), c[1] + d * math.sin(a)
            b = rng.uniform(0, math.pi)
            hl = rng.uniform(0.06, 0.12) * s
            spec.holes.append(("slot", px - hl * math.cos(b), py - hl * math.sin(b),
                               px + hl * math.cos(b), py + hl * math.sin(b), rng.uniform(0.025, 0.04) * s))
    else:
        raise ValueError(kind)
    return spec


# ----------------------------------------------------------------------------
# rendering
# ----------------------------------------------------------------------------

def _round_u8(v):
    return np.clip(np.floor(v + 0.5), 0, 255).astype(np.uint8)


def render_template(spec: PartSpec) -> np.ndarray:
    """The template image: part at part_level on background, 4x4 supersampled."""
    h, w = spec.height, spec.width
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    acc = np.zeros((h, w), dtype=np.float64)
    for oy in _SUB:
        for ox in _SUB:
            m = spec.inside(xs + ox, ys + oy)
            acc += np.where(m, spec.part_level, spec.background)
    return _round_u8(acc / 16.0)


def _inverse_map(qx, qy, pose, spec):
    ux, uy, th = pose[:3]
    sc = pose[3] if len(pose) > 3 else 1.0     # optional scale of the instance
    c, s = math.cos(math.radians(th)), math.sin(math.radians(th))
    dx, dy = (qx - ux) / sc, (qy - uy) / sc
    tx = c * dx + s * dy + spec.width // 2
    ty = -s * dx + c * dy + spec.height // 2
    return tx, ty


def _exact_quarter_turn(th):
    q = th / 90.0
    return abs(q - round(q)) < 1e-12


def _quarter_cos_sin(th):
    k = int(round(th / 90.0)) % 4
    return [(1, 0), (0, 1), (-1, 0), (0, -1)][k]


def render_scene(bg: np.ndarray, instances, paste_square=False) -> np.ndarray:
    """Render instances onto a float background (H x W) and return float64.

    instances: list of (spec, (u_x, u_y, theta_deg), level) where level is the
    intensity of the part body (None keeps spec.part_level).  With
    paste_square=True the template's own background square is drawn too
    (a pasted template); otherwise only the part body is drawn and the
    scene background shows through holes and around the part.
    """
    out = bg.astype(np.float64).copy()
    H, W = out.shape
    for spec, pose, level in instances:
        part_level = spec.part_level if level is None else level
        ux, uy, th = pose[:3]
        sc = pose[3] if len(pose) > 3 else 1.0
        rad = 0.5 * math.hypot(spec.width, spec.height) * sc + 2
        x0, x1 = max(0, int(math.floor(ux - rad))), min(W, int(math.ceil(ux + rad)) + 1)
        y0, y1 = max(0, int(math.floor(uy - rad))), min(H, int(math.ceil(uy + rad)) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        ys, xs = np.mgrid[y0:y1, x0:x1].astype(np.float64)
        acc = np.zeros(xs.shape, dtype=np.float64)
        cover = np.zeros(xs.shape, dtype=np.float64)
        quarter = _exact_quarter_turn(th) and float(ux).is_integer() and float(uy).is_integer() and sc == 1.0
        for oy in _SUB:
            for ox in _SUB:
                qx, qy = xs + ox, ys + oy
                if quarter:
                    # exact integer-friendly inverse map for quarter turns
                    c, s = _quarter_cos_sin(th)
                    dx, dy = qx - ux, qy - uy
                    tx = c * dx + s * dy + spec.width // 2
                    ty = -s * dx + c * dy + spec.height // 2
                else:
                    tx, ty = _inverse_map(qx, qy, pose, spec)
                m = spec.inside(tx, ty)
                if paste_square:
                    sq = spec.on_template(tx, ty)
                    val = np.where(m, part_level, spec.background)
                    acc += np.where(sq, val, 0.0)
                    cover += sq
                else:
                    acc += np.where(m, part_level, 0.0)
                    cover += m
        region = out[y0:y1, x0:x1]
        out[y0:y1, x0:x1] = region * (1.0 - cover / 16.0) + acc / 16.0
    return out


def _segment_mask(H, W, ax, ay, bx, by, r):
    """Coverage of a thick segment, as (y0, x0, local array) over its box."""
    x0, x1 = max(0, int(min(ax, bx) - r - 1)), min(W, int(max(ax, bx) + r + 2))
    y0, y1 = max(0, int(min(ay, by) - r - 1)), min(H, int(max(ay, by) + r + 2))
    if x0 >= x1 or y0 >= y1:
        return 0, 0, np.zeros((0, 0))
    ys, xs = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    acc = np.zeros(xs.shape)
    for oy in _SUB:
        for ox in _SUB:
            acc += _in_prim(xs + ox, ys + oy, ("slot", ax, ay, bx + 1e-9, by, r))
    return y0, x0, acc / 16.0


def _rect_cover(H, W, cx, cy, hw, hh, ang):
    """Coverage of a rotated rectangle, as (y0, x0, local array) over its box."""
    rad = math.hypot(hw, hh) + 2
    x0, x1 = max(0, int(cx - rad)), min(W, int(cx + rad) + 1)
    y0, y1 = max(0, int(cy - rad)), min(H, int(cy + rad) + 1)
    if x0 >= x1 or y0 >= y1:
        return 0, 0, np.zeros((0, 0))
    ys, xs = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    c, s = math.cos(ang), math.sin(ang)
    acc = np.zeros(xs.shape)
    for oy in _SUB:
        for ox in _SUB:
            dx, dy = xs + ox - cx, ys + oy - cy
            lx, ly = c * dx + s * dy, -s * dx + c * dy
            acc += (np.abs(lx) < hw) & (np.abs(ly) < hh)
    return y0, x0, acc / 16.0


def _blend(img, cover, g):
    """Paint grey level g over img with the given local coverage, in place."""
    y0, x0, cov = cover
    h, w = cov.shape
    if h and w:
        region = img[y0:y0 + h, x0:x0 + w]
        img[y0:y0 + h, x0:x0 + w] = region * (1 - cov) + g * cov
    return img


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def paste_scene(spec, size, poses, background=60.0):
    """Noise-free scene of constant background with the template pasted at poses."""
    W, H = size
    bg = np.full((H, W), background, dtype=np.float64)
    inst = [(spec, p, None) for p in poses]
    return _round_u8(render_scene(bg, inst, paste_square=True))


def tiny_case(seed, size=32, tsize=9):
    """A small random template and a small random search image (brute-force sizes)."""
    rng = np.random.default_rng(seed)
    spec = random_part(rng, tsize, kind="tiny", margin=1.0)
    tmpl = render_template(spec)
    H = W = size
    bg = rng.normal(110.0, 20.0, (H, W))
    poses = [(int(rng.integers(2, W - 2)), int(rng.integers(2, H - 2)), float(rng.uniform(0, 360)))]
    scene = render_scene(bg, [(spec, poses[0], None)], paste_square=True)
    scene += rng.normal(0.0, 4.0, scene.shape)
    return tmpl, _round_u8(scene), poses


def config1_scene(seed=2234):
    """320x240, 3 pasted 48x48 templates (polygon + ring, 200 on 60) on N(110, 8^2)."""
    rng = np.random.default_rng(seed)
    spec = random_part(rng, 48, kind="tiny", margin=3.0)
    tmpl = render_template(spec)
    W, H = 320, 240
    bg = rng.normal(110.0, 8.0, (H, W))
    poses = []
    tries = 0
    while len(poses) < 3 and tries < 1000:
        tries += 1
        p = (int(rng.integers(30, W - 30)), int(rng.integers(30, H - 30)), float(rng.uniform(0, 360)))
        if all(math.hypot(p[0] - q[0], p[1] - q[1]) > 70 for q in poses):
            poses.append(p)
    scene = render_scene(bg, [(spec, p, None) for p in poses], paste_square=True)
    return tmpl, _round_u8(scene), poses


def _scene_background(rng, H, W, level=100.0):
    return np.full((H, W), level, dtype=np.float64)


def config2_scene(seed=3234, W=1280, H=1024, side=200, spec=None, n_inst=None, subpixel=False, scales=None):
    """Paper-shaped scene: 1-4 instances of a side x side part with occlusion,
    an illumination ramp, 20 clutter segments and Gaussian noise sigma=6.

    Returns (template uint8, scene uint8, ground-truth poses, spec).
    Instance angles are drawn on a 0.5 degree grid, positions on the pixel
    grid; with subpixel=True each position is moved by U(-1/2, 1/2) px per
    axis, drawn from a second generator so the scene is otherwise the same.
    With `scales` (a list) each instance is drawn at a scale chosen from it
    by a third generator (poses then carry it: (x, y, theta, s)), and the
    placement keeps the largest scale's extent inside the image.
    """
    rng = np.random.default_rng(seed)
    if spec is None:
        spec = random_part(rng, side, kind="part", margin=4.0)
    tmpl = render_template(spec)
    bg = _scene_background(rng, H, W, level=float(rng.uniform(80, 110)))
    if n_inst is None:
        n_inst = int(rng.integers(1, 5))
    poses = []
    tries = 0
    rad = 0.5 * math.hypot(side, side) * (max(scales) if scales else 1.0)
    while len(poses) < n_inst and tries < 10000:
        tries += 1
        p = (int(rng.integers(int(rad * 0.6), W - int(rad * 0.6))),
             int(rng.integers(int(rad * 0.6), H - int(rad * 0.6))),
             0.5 * float(rng.integers(0, 720)))
        if all(math.hypot(p[0] - q[0], p[1] - q[1]) > 1.5 * rad for q in poses):
            poses.append(p)
    if subpixel:
        frac = np.random.default_rng(seed + 0x5EED).uniform(-0.5, 0.5, (len(poses), 2))
        poses = [(p[0] + float(f[0]), p[1] + float(f[1]), p[2]) for p, f in zip(poses, frac)]
    if scales:
        pick = np.random.default_rng(seed + 0x5CA1E).integers(0, len(scales), len(poses))
        poses = [(p[0], p[1], p[2], float(scales[int(i)])) for p, i in zip(poses, pick)]
    img = render_scene(bg, [(spec, p, float(rng.uniform(170, 210))) for p in poses])
    # clutter: 20 random line segments, 1.5-3 px thick, random gray
    for _ in range(20):
        ax, ay = rng.uniform(0, W), rng.uniform(0, H)
        L = rng.uniform(30, 200)
        a = rng.uniform(0, 2 * math.pi)
        cov = _segment_mask(H, W, ax, ay, ax + L * math.cos(a), ay + L * math.sin(a), rng.uniform(0.75, 1.5))
        g = rng.uniform(20, 240)
        img = _blend(img, cov, g)
    # occluders: rectangles covering 0-40 % of each instance
    for p in poses:
        frac = rng.uniform(0.0, 0.4)
        if frac < 0.02:
            continue
        area = frac * side * side
        aspect = rng.uniform(0.5, 2.0)
        hw = 0.5 * math.sqrt(area * aspect)
        hh = 0.5 * math.sqrt(area / aspect)
        off = rng.uniform(0.3, 0.6) * side
        a = rng.uniform(0, 2 * math.pi)
        cov = _rect_cover(H, W, p[0] + off * math.cos(a), p[1] + off * math.sin(a), hw, hh, rng.uniform(0, math.pi))
        g = rng.uniform(20, 240)
        img = _blend(img, cov, g)
    # illumination ramp: gain linear across the image along a random direction
    g0, g1 = rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.5)
    off = rng.uniform(-40, 40)
    a = rng.uniform(0, 2 * math.pi)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    proj = (xs - W / 2) * math.cos(a) + (ys - H / 2) * math.sin(a)
    t = (proj - proj.min()) / max(1e-9, proj.max() - proj.min())
    img = img * (g0 + (g1 - g0) * t) + off
    img = img + rng.normal(0.0, 6.0, img.shape)
    return tmpl, _round_u8(img), poses, spec


def config3_batch(seed=4234, n_images=64, sizes=((640, 480), (1280, 1024), (1920, 1080), (2592, 1944)),
                  sides=(64, 96, 128, 200, 256, 320, 384, 400)):
    """Uneven batch: templates of the given sides, images of random sizes,
    each image matched against 2 templates (pairs list of (image, template)).
    """
    rng = np.random.default_rng(seed)
    specs = [random_part(rng, s, kind="part", margin=4.0) for s in sides]
    tmpls = [render_template(s) for s in specs]
    images, pairs, truth = [], [], []
    for i in range(n_images):
        W, H = sizes[int(rng.integers(0, len(sizes)))]
        ts = rng.choice(len(sides), size=2, replace=False)
        fits = [int(t) for t in ts if sides[t] * 1.5 < min(W, H)]
        if not fits:
            fits = [0]
        spec = specs[fits[0]]
        _, img, poses, _ = config2_scene(seed=int(rng.integers(0, 2**31)), W=W, H=H, side=spec.width,
                                         spec=spec, n_inst=int(rng.integers(1, 3)))
        images.append(img)
        truth.append((fits[0], poses))
        for t in ts:
            pairs.append((i, int(t)))
    return tmpls, images, pairs, truth


def config4_triples(seed=5234, n=4096, n_scenes=4):
    """Pose-refinement triples: (scene index, ground truth, perturbed initial pose)."""
    rng = np.random.default_rng(seed)
    scenes = []
    spec = None
    tmpl = None
    for k in range(n_scenes):
        t, img, poses, spec = config2_scene(seed=seed + 17 * k, spec=spec)
        tmpl = t if tmpl is None else tmpl
        scenes.append((img, poses))
    triples = []
    for _ in range(n):
        k = int(rng.integers(0, n_scenes))
        gt = scenes[k][1][int(rng.integers(0, len(scenes[k][1])))]
        init = (gt[0] + rng.uniform(-1.5, 1.5), gt[1] + rng.uniform(-1.5, 1.5), gt[2] + rng.uniform(-1.5, 1.5))
        triples.append((k, gt, init))
    return tmpl, [s[0] for s in scenes], triples


def config5_scene(seed=6234, W=4096, H=3072, side=512):
    """Large stress scene: 6 instances of a 512x512 part, 30 % occlusion."""
    rng = np.random.default_rng(seed)
    spec = random_part(rng, side, kind="part", margin=6.0)
    tmpl, img, poses, _ = config2_scene(seed=seed + 1, W=W, H=H, side=side, spec=spec, n_inst=6)
    return tmpl, img, poses

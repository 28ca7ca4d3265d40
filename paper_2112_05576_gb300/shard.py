"""Host logic of a search sharded over ranks (one process per GPU).

Two ways to split the exhaustive search of Sec. II over ranks:

* independent units (images, (image, template) pairs): each rank takes a
  contiguous share of the units and nothing is exchanged (`unit_range`);
* one large search split by angle block: rank r scores the angles of its
  block plus one halo angle on each side (theta is circular), extracts the
  strict local maxima of its own angles -- the halo planes supply the
  neighbours across the block boundary -- and the ranks exchange only their
  top-K candidate lists (an all-gather of K x 16 bytes per rank); every rank
  then merges the lists in the same total order (higher score, then smaller
  key (k * H + y) * W + x) and so holds the same global top-K as a
  single-rank search.

The per-rank scoring and candidate extraction are passed in as callables;
`gpu_score_fn` and `gpu_candidates_fn` are the library's (sam_score_window
and sam_candidates).  Only argument marshalling and the merge of the
exchanged lists run on the host.
"""

from __future__ import annotations

from typing import Callable, List, Sequence, Tuple

import numpy as np

Cand = Tuple[int, int, int, float]   # (k, y, x, score), k global


def unit_range(n_units: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous share [begin, end) of n_units for `rank` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_units, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def angle_block(nth: int, world: int, rank: int) -> Tuple[int, int]:
    """(k0, nk) of rank's angle block; every rank gets at least one angle."""
    if world > nth:
        raise ValueError("more ranks than angles")
    b, e = unit_range(nth, world, rank)
    return b, e - b


def extended_angles(k0: int, nk: int, nth: int) -> List[int]:
    """Global angle indices of a block with one halo angle on each side (the
    whole circle, unextended, when the block is all angles)."""
    if nk == nth:
        return list(range(nth))
    return [(k0 - 1) % nth] + list(range(k0, k0 + nk)) + [(k0 + nk) % nth]


def contiguous_runs(angles: Sequence[int]) -> List[Tuple[int, int, int]]:
    """Split a list of angle indices into runs (position, k0, count) of
    consecutive indices (what one windowed scoring call can serve)."""
    runs = []
    i = 0
    while i < len(angles):
        j = i
        while j + 1 < len(angles) and angles[j + 1] == angles[j] + 1:
            j += 1
        runs.append((i, angles[i], j - i + 1))
        i = j + 1
    return runs


def order_key(c: Cand, H: int, W: int):
    k, y, x, s = c
    return (-s, (k * H + y) * W + x)


def merge_candidates(lists: Sequence[Sequence[Cand]], K: int, H: int, W: int) -> List[Cand]:
    """Global top-K of per-rank candidate lists under the detector's total order."""
    allc = [tuple(c) for lst in lists for c in lst]
    allc.sort(key=lambda c: order_key(c, H, W))
    return [(int(k), int(y), int(x), float(s)) for k, y, x, s in allc[:K]]


def block_candidates(k0: int, nk: int, nth: int, H: int, W: int, min_score: float, K: int,
                     score_fn: Callable, cand_fn: Callable) -> List[Cand]:
    """This rank's top-K strict local maxima over its own angles.

    score_fn(k_first, count) -> array (count, H, W) of scores of angles
    k_first .. k_first + count - 1; cand_fn(map, min_score, K) -> (k, y, x, s)
    arrays of the best K strict local maxima of a map whose planes are
    circular.  The halo planes only serve as neighbours: their own maxima are
    dropped, and K is raised until K maxima of the block's own planes are
    certain to be among those returned.
    """
    # The block and its halo planes, in increasing global angle index: a
    # block that wraps around angle 0 ([nth-1, 0, 1, ..]) is stored as
    # [0, 1, .., nth-1], so the extended map's circular plane order keeps every
    # own plane next to its two global neighbours, and its plane order is the
    # global one, so cand_fn breaks ties between planes as the single-rank
    # search does (higher score, then the smaller global key).
    ext = sorted(set(extended_angles(k0, nk, nth)))
    planes = []
    for _, ka, cnt in contiguous_runs(ext):
        planes.append(score_fn(ka, cnt))
    emap = planes[0] if len(planes) == 1 else _concat(planes)
    halo = len(ext) != nth

    def is_own(g):
        return (g - k0) % nth < nk

    k_ext = K if not halo else 4 * K
    while True:
        ks, ys, xs, ss = cand_fn(emap, min_score, k_ext)
        own = [(ext[int(k)], int(y), int(x), float(s)) for k, y, x, s in zip(ks, ys, xs, ss)
               if not halo or is_own(ext[int(k)])]
        if len(own) >= K or len(ks) < k_ext:
            own.sort(key=lambda c: order_key(c, H, W))
            return own[:K]
        k_ext *= 2


def _concat(planes):
    try:
        import torch
        if isinstance(planes[0], torch.Tensor):
            return torch.cat(planes, dim=0)
    except ImportError:
        pass
    return np.concatenate(planes, axis=0)


def sharded_candidates(nth: int, H: int, W: int, min_score: float, K: int, score_fn: Callable,
                       cand_fn: Callable, group=None) -> List[Cand]:
    """The global top-K candidates of a search split by angle block over the
    ranks of `group` (torch.distributed; world 1 without it).  Identical on
    every rank."""
    world, rank = 1, 0
    if group is not None or _dist_ready():
        import torch.distributed as dist
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    k0, nk = angle_block(nth, world, rank)
    mine = block_candidates(k0, nk, nth, H, W, min_score, K, score_fn, cand_fn)
    if world == 1:
        return merge_candidates([mine], K, H, W)
    import torch.distributed as dist
    lists = [None] * world
    dist.all_gather_object(lists, mine, group=group)
    return merge_candidates(lists, K, H, W)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The maximum of a per-rank number (a timed region's milliseconds) over
    the ranks of `group`; the value itself without torch.distributed."""
    if group is None and not _dist_ready():
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def whole_job_rate(units_per_rank_step: float, steps: int, world: int, ms_max: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest
    rank's time (weak scaling: the per-rank work is fixed)."""
    return units_per_rank_step * steps * world / (ms_max * 1e-3)


def _dist_ready():
    try:
        import torch.distributed as dist
        return dist.is_available() and dist.is_initialized()
    except ImportError:
        return False


# ---------------------------------------------------------------------------
# the library's per-rank steps
# ---------------------------------------------------------------------------

def gpu_score_fn(model, level, field, w, h, precision, nbhd=3, min_score=0.0, early=0):
    """score_fn over the library's windowed scorer (whole translation range)."""
    import torch

    from . import sam

    def fn(k_first, count):
        out = torch.empty((count, h, w), dtype=torch.float32, device=field.device)
        sam.score_window(model, level, field, w, h, precision, 0, 0, w, h, k_first, count, out, nbhd=nbhd,
                         min_score=min_score, early=early)
        return out

    return fn


def gpu_candidates_fn():
    """cand_fn over the library's candidate kernels."""
    import torch

    from . import sam

    def fn(smap, min_score, K):
        nth, gh, gw = smap.shape
        dev = smap.device
        kyx = torch.empty((K, 3), dtype=torch.int32, device=dev)
        s = torch.empty(K, dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        scratch = torch.empty(sam.candidates_scratch_bytes(nth, gh, gw), dtype=torch.uint8, device=dev)
        sam.candidates(smap.contiguous(), min_score, K, kyx, s, cnt, scratch)
        n = int(cnt.item())
        kyx = kyx[:n].cpu().numpy()
        return kyx[:, 0], kyx[:, 1], kyx[:, 2], s[:n].cpu().numpy()

    return fn

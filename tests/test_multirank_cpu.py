"""Multi-rank host logic on CPU ranks (torch.distributed, gloo).

A search split by angle block over 2 or 3 ranks, with the FP64 oracle as
each rank's scorer and candidate extractor, must give exactly the global
top-K candidates of a single-rank search (same poses, same scores, same
order); the benchmark's timing aggregation (max over ranks, whole-job rate)
and the unit split are checked on the same ranks.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_2112_05576_gb300 import shard  # noqa: E402

MIN_SCORE = 0.3
K = 12
STEP = 10.0


def _case():
    tmpl, img, _ = synth.tiny_case(5, size=48, tsize=13)
    om = oracle.create_model(tmpl, 30, 60, 1, STEP)
    field = oracle.search_fields(img, 1, 30)[0]
    return om, field


def _oracle_fns(om, field):
    def score_fn(k_first, count):
        return oracle.score_map_range(field, om.points[0], k_first, count, STEP, nbhd=3)

    def cand_fn(smap, min_score, k):
        return oracle.candidates(smap, min_score, k)

    return score_fn, cand_fn


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        om, field = _case()
        H, W = field.shape[:2]
        nth = om.ntheta(0)
        score_fn, cand_fn = _oracle_fns(om, field)
        got = shard.sharded_candidates(nth, H, W, MIN_SCORE, K, score_fn, cand_fn)
        # timing aggregation: rank r reports 10 + r ms
        ms = shard.max_over_ranks(10.0 + rank)
        rate = shard.whole_job_rate(1000.0, 5, world, ms)
        lists = [None] * world
        dist.all_gather_object(lists, (got, ms, rate, shard.angle_block(nth, world, rank)))
        if rank == 0:
            out.put(lists)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_angle_sharded_candidates_equal_single_rank(world):
    om, field = _case()
    H, W = field.shape[:2]
    nth = om.ntheta(0)
    full = oracle.score_map(field, om.points[0], nth, STEP, nbhd=3)
    ks, ys, xs, ss = oracle.candidates(full, MIN_SCORE, K)
    want = [(int(k), int(y), int(x), float(s)) for k, y, x, s in zip(ks, ys, xs, ss)]
    assert len(want) >= 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    lists = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for got, ms, rate, blk in lists:
        assert got == want                      # every rank holds the global top-K
        assert ms == 10.0 + (world - 1)         # max over ranks
        assert rate == pytest.approx(1000.0 * 5 * world / (ms * 1e-3))
    blocks = sorted(l[3] for l in lists)
    assert blocks[0][0] == 0 and sum(b[1] for b in blocks) == nth
    assert all(blocks[i][0] + blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))


def test_single_rank_block_is_the_whole_circle():
    om, field = _case()
    H, W = field.shape[:2]
    nth = om.ntheta(0)
    score_fn, cand_fn = _oracle_fns(om, field)
    got = shard.sharded_candidates(nth, H, W, MIN_SCORE, K, score_fn, cand_fn)
    ks, ys, xs, ss = oracle.candidates(oracle.score_map(field, om.points[0], nth, STEP, nbhd=3), MIN_SCORE, K)
    assert got == [(int(k), int(y), int(x), float(s)) for k, y, x, s in zip(ks, ys, xs, ss)]


def test_unit_ranges_and_halo():
    for n in [0, 1, 7, 64, 128]:
        for world in [1, 2, 3, 8]:
            rs = [shard.unit_range(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            assert max(e - b for b, e in rs) - min(e - b for b, e in rs) <= 1
    assert shard.extended_angles(0, 3, 36) == [35, 0, 1, 2, 3]
    assert shard.extended_angles(33, 3, 36) == [32, 33, 34, 35, 0]
    assert shard.extended_angles(0, 36, 36) == list(range(36))
    assert shard.contiguous_runs([35, 0, 1, 2, 3]) == [(0, 35, 1), (1, 0, 4)]
    with pytest.raises(ValueError):
        shard.angle_block(4, 5, 0)


# ---------------------------------------------------------------------------
# exact ties across block boundaries and across the angle wrap
# ---------------------------------------------------------------------------

TIE_NTH, TIE_H, TIE_W = 12, 6, 7


def _tied_map():
    # multiples of 1/8: many exact ties between neighbouring planes, and the
    # first and last planes made equal so that ties straddle the wrap
    rng = np.random.default_rng(77)
    m = rng.integers(0, 9, (TIE_NTH, TIE_H, TIE_W)) / 8.0
    m[-1] = m[0]
    m[5] = m[6]
    return m


def _tied_fns():
    full = _tied_map()

    def score_fn(k_first, count):
        return full[k_first:k_first + count]

    def cand_fn(smap, min_score, k):
        return oracle.candidates(smap, min_score, k)

    return score_fn, cand_fn


def _tie_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        score_fn, cand_fn = _tied_fns()
        got = shard.sharded_candidates(TIE_NTH, TIE_H, TIE_W, 0.25, 40, score_fn, cand_fn)
        lists = [None] * world
        dist.all_gather_object(lists, got)
        if rank == 0:
            out.put(lists)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_sharded_candidates_break_ties_as_single_rank(world):
    ks, ys, xs, ss = oracle.candidates(_tied_map(), 0.25, 40)
    want = [(int(k), int(y), int(x), float(s)) for k, y, x, s in zip(ks, ys, xs, ss)]
    assert len(want) >= 10
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tie_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    lists = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for got in lists:
        assert got == want


def test_block_candidates_with_ties_without_processes():
    # every block of every split, checked in one process against the single-rank search
    score_fn, cand_fn = _tied_fns()
    ks, ys, xs, ss = oracle.candidates(_tied_map(), 0.25, 40)
    want = [(int(k), int(y), int(x), float(s)) for k, y, x, s in zip(ks, ys, xs, ss)]
    for world in (2, 3, 4, 6, 12):
        lists = []
        for r in range(world):
            k0, nk = shard.angle_block(TIE_NTH, world, r)
            lists.append(shard.block_candidates(k0, nk, TIE_NTH, TIE_H, TIE_W, 0.25, 40, score_fn, cand_fn))
        assert shard.merge_candidates(lists, 40, TIE_H, TIE_W) == want, world

"""The allocation-free candidate entry point against the regular one and the oracle.

sam_candidates_noalloc serves callers that cannot call cudaMalloc when they
need candidates (deadline-bound loops, fixed device-memory budgets); it must
give exactly what sam_candidates gives with a caller-provided scratch
buffer, call after call, since its own scratch persists between calls, and
exactly what the oracle's candidate selection gives on the same map (the
maps hold multiples of 1/8, so FP32 and FP64 order them alike).
Collected last so a failure here cannot hide any other test's result.
"""

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2112_05576_gb300 as sam  # noqa: E402
from paper_2112_05576_gb300 import sam as samb  # noqa: E402


def _run(fn, smap, K, **kw):
    kyx = torch.full((3 * K,), -7, dtype=torch.int32, device="cuda")
    s = torch.full((K,), -7.0, dtype=torch.float32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    fn(smap, 0.5, K, kyx, s, cnt, **kw)
    torch.cuda.synchronize()
    n = int(cnt.item())
    return n, kyx.cpu().numpy()[: 3 * n].copy(), s.cpu().numpy()[:n].copy()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_noalloc_matches_regular_entry_point_twice():
    rng = np.random.default_rng(2112)
    K = 64
    # two different maps of the size of a 1280x1024 search's top level
    maps = [torch.from_numpy((rng.integers(0, 9, (45, 128, 160)) / 8.0).astype(np.float32)).cuda()
            for _ in range(2)]
    for smap in maps:       # two calls in a row on the shared device scratch
        nth, gh, gw = smap.shape
        scratch = torch.empty(sam.candidates_scratch_bytes(nth, gh, gw), dtype=torch.uint8, device="cuda")
        ref = _run(sam.candidates, smap, K, scratch=scratch)
        got = _run(samb.candidates_noalloc, smap, K)
        assert ref[0] > 0 and got[0] == ref[0]
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])
        ck, cy, cx, cs = oracle.candidates(smap.cpu().numpy().astype(np.float64), 0.5, K)
        assert got[0] == len(ck)
        kyx = got[1].reshape(-1, 3)
        assert np.array_equal(kyx[:, 0], ck) and np.array_equal(kyx[:, 1], cy) and np.array_equal(kyx[:, 2], cx)
        assert np.array_equal(got[2], cs.astype(np.float32))


def test_noalloc_rejects_maps_beyond_its_scratch():
    big = torch.zeros((360, 256, 512), dtype=torch.float32, device="cuda")   # needs ~94 MB of scratch
    with pytest.raises(sam.SamError) as e:
        _run(samb.candidates_noalloc, big, 8)
    assert e.value.status == samb.SAM_ERR_CAPACITY

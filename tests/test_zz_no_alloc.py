"""The allocation-free hypervolume entry point, for callers that cannot allocate device
memory when they need the result (their device memory belongs to another allocator, or
an allocation would stall the device). Its scratch is a fixed array inside the library,
shared by every call. Checked through the C ABI against the allocating entry point,
which takes a caller-provided workspace, on consecutive calls; hypervolumes are exact
integers, so the two must agree exactly. Collected last on purpose."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_2604_26477_b300 import build
    build.build()
    from paper_2604_26477_b300 import moqaia
    return moqaia


def _points(seed, F, K, span):
    rng = np.random.default_rng(seed)
    pts = rng.integers(-span // 10, span, size=(F, K)).astype(np.int64)
    pts[: F // 2, -1] = 2 * span - pts[: F // 2, :-1].sum(axis=1)  # mostly non-dominated
    return pts


def _with_workspace(M, pts_dev, F, K, ref):
    ws = torch.zeros(M.moq_hypervolume_workspace_size(F, K), dtype=torch.uint8, device="cuda")
    return M.moq_hypervolume_points(pts_dev, F, K, ref, ws)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(M):
    cases = [(1, 1800, 3, 500), (2, 400, 4, 60), (3, 37, 3, 1000), (4, 5000, 2, 10**6)]
    for seed, F, K, span in cases:  # larger and smaller sets in a row: stale scratch must not leak
        pts = _points(seed, F, K, span)
        ref = np.zeros(K, np.int64)
        dev = torch.from_numpy(pts).cuda()
        want = _with_workspace(M, dev, F, K, ref)
        first = M.moq_hypervolume_points_noalloc(dev, F, K, ref)
        second = M.moq_hypervolume_points_noalloc(dev, F, K, ref)
        assert first == want and second == want
    assert M.moq_hypervolume_points_noalloc(torch.zeros((1, 3), dtype=torch.int64, device="cuda"), 0, 3,
                                            np.zeros(3, np.int64)) == 0


def test_noalloc_from_a_fresh_host_thread(M):
    # a host thread that never called the library before: the result comes back into the
    # call's own stack frame, not a per-thread pinned buffer created on first use
    import threading
    pts = _points(5, 900, 3, 700)
    ref = np.zeros(3, np.int64)
    dev = torch.from_numpy(pts).cuda()
    want = _with_workspace(M, dev, 900, 3, ref)
    got = {}

    def run():
        try:
            got["hv"] = [M.moq_hypervolume_points_noalloc(dev, 900, 3, ref) for _ in range(2)]
        except Exception as e:  # surfaced by the assertion below
            got["err"] = e

    t = threading.Thread(target=run)
    t.start()
    t.join(120)
    assert "err" not in got, got.get("err")
    assert got["hv"] == [want, want]


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(M):
    limit = M.moq_hypervolume_noalloc_max_points()
    assert limit == 16384
    pts = torch.zeros((limit + 1, 3), dtype=torch.int64, device="cuda")
    with pytest.raises(M.MoqError) as e:
        M.moq_hypervolume_points_noalloc(pts, limit + 1, 3, np.zeros(3, np.int64))
    assert e.value.code == M.MOQ_ERR_CAPACITY and "limit" in str(e.value)
    # exactly at the limit, four objectives (the streamed slab kernels): the whole array in use
    full = _points(6, limit, 4, 90)
    ref = np.zeros(4, np.int64)
    dev = torch.from_numpy(full).cuda()
    assert M.moq_hypervolume_points_noalloc(dev, limit, 4, ref) == _with_workspace(M, dev, limit, 4, ref)

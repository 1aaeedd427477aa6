"""bf_search_noalloc: the brute-force search for callers that cannot allocate
device memory (its scratch is a static array inside the library).  Checked
through the C ABI against bf_search and against the FP64 oracle, on two calls
in a row, with the tolerance of the other parity tests, and at the edges of
its documented size limits.  Collected last so that a stop-at-first-failure
run has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from parity import DIST_REL, check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

SCRATCH = 32 << 20
HEAD = 256


def _entry():
    f = rbc.load().bf_search_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _call(f, Q, X, k, metric, ids=None, dist=None):
    m, d = Q.shape
    if ids is None:
        ids = torch.full((m, k), -7, dtype=torch.int64, device="cuda")
        dist = torch.full((m, k), -7.0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(Q.data_ptr(), m, X.data_ptr(), X.shape[0], d, k, metric, ids.data_ptr(),
           dist.data_ptr(), stream)
    return rc, ids, dist


def max_queries(k):
    """Largest m the documented limit admits: ceil(m / 128) tiles of
    128 x 2 x C x 8-byte lists plus 4 m bytes (rounded up to 256) after the
    256-byte head, C the smallest of 2 .. 32 that is >= k + 1."""
    C = next(c for c in (2, 4, 8, 16, 32) if c >= k + 1)

    def fits(m):
        rows = (4 * m + 255) // 256 * 256
        return -(-m // 128) * 128 * 2 * C * 8 + rows <= SCRATCH - HEAD

    lo, hi = 1, 1 << 22
    while lo < hi:
        mid = (lo + hi + 1) // 2
        lo, hi = (mid, hi) if fits(mid) else (lo, mid - 1)
    return lo


def test_documented_limits():
    # the numbers stated in rbc.h
    assert [max_queries(k) for k in (1, 2, 4, 8, 16)] == [931968, 493440, 254080, 129024, 65024]


def test_noalloc_matches_bf_search_and_oracle_on_two_calls():
    f = _entry()
    cases = [(50000, 3000, 64, 10, rbc.L2, 1), (20011, 777, 33, 5, rbc.L1, 2),
             (4096, 300, 33, 1, rbc.L2, 3), (4096, 300, 33, 10, rbc.L1, 4)]
    for n, m, d, k, metric, seed in cases:
        Xh = synth.iid_normal(n, d, 100 + seed)
        Qh = synth.iid_normal(m, d, 200 + seed)
        X, Q = torch.from_numpy(Xh).cuda(), torch.from_numpy(Qh).cuda()
        ref_ids, ref_dist = rbc.bf_search(Q, X, k, metric=metric, storage=rbc.F32)
        ref_ids, ref_dist = ref_ids.cpu().numpy(), ref_dist.cpu().numpy()
        o_ids, o_rho = oracle.bf(Qh, Xh, k, "l2" if metric == rbc.L2 else "l1")
        for _ in range(2):  # the scratch keeps the previous call's contents
            rc, ids, dist = _call(f, Q, X, k, metric)
            assert rc == 0, rbc.load().rbc_last_error().decode()
            torch.cuda.synchronize()
            ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
            np.testing.assert_array_equal(ids, ref_ids)
            a, b = dist.astype(np.float64), ref_dist.astype(np.float64)
            assert np.all(np.abs(a - b) <= DIST_REL * np.maximum(b, 1e-30))
            check_knn(Qh, Xh, ids, dist, o_ids, o_rho, "l2" if metric == rbc.L2 else "l1")
            st = rbc.last_stats()
            assert st["queries"] == m


@pytest.mark.parametrize("k", [10, 16])
def test_noalloc_size_limit_edges(k):
    f = _entry()
    mmax = max_queries(k)
    X = torch.from_numpy(synth.iid_normal(64, 8, 5)).cuda()
    Q = torch.from_numpy(synth.iid_normal(mmax + 1, 8, 6)).cuda()
    ids = torch.empty((mmax + 1, k), dtype=torch.int64, device="cuda")
    dist = torch.empty((mmax + 1, k), dtype=torch.float32, device="cuda")
    rc, _, _ = _call(f, Q, X, k, rbc.L2, ids, dist)
    assert rc == -5
    assert "scratch" in rbc.load().rbc_last_error().decode()
    rc, _, _ = _call(f, Q[:mmax], X, k, rbc.L2, ids, dist)
    assert rc == 0, rbc.load().rbc_last_error().decode()
    torch.cuda.synchronize()
    sample = np.arange(0, mmax, 997)
    o_ids, o_rho = oracle.bf(Q[sample].cpu().numpy(), X.cpu().numpy(), k, "l2")
    check_knn(Q[sample].cpu().numpy(), X.cpu().numpy(), ids[sample].cpu().numpy(),
              dist[sample].cpu().numpy(), o_ids, o_rho, "l2")


def test_noalloc_rejects_host_buffers():
    f = _entry()
    X = np.zeros((64, 8), np.float32)
    Q = np.zeros((4, 8), np.float32)
    ids = np.empty((4, 2), np.int64)
    dist = np.empty((4, 2), np.float32)
    rc = f(Q.ctypes.data, 4, X.ctypes.data, 64, 8, 2, rbc.L2, ids.ctypes.data, dist.ctypes.data, None)
    assert rc == -1

"""bf_search_noalloc: the brute-force search for callers that cannot allocate
device memory (its scratch is a static array inside the library).  Checked
through the C ABI against bf_search, on two calls in a row, with the tolerance
of the other parity tests.  Collected last so that a stop-at-first-failure run
has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth
from parity import DIST_REL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402


def _entry():
    f = rbc.load().bf_search_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_matches_bf_search_on_two_calls():
    f = _entry()
    cases = [(50000, 3000, 64, 10, rbc.L2, 1), (20011, 777, 33, 5, rbc.L1, 2)]
    for n, m, d, k, metric, seed in cases:
        X = torch.from_numpy(synth.iid_normal(n, d, 100 + seed)).cuda()
        Q = torch.from_numpy(synth.iid_normal(m, d, 200 + seed)).cuda()
        ref_ids, ref_dist = rbc.bf_search(Q, X, k, metric=metric, storage=rbc.F32)
        ids = torch.full((m, k), -7, dtype=torch.int64, device="cuda")
        dist = torch.full((m, k), -7.0, dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = f(Q.data_ptr(), m, X.data_ptr(), n, d, k, metric, ids.data_ptr(), dist.data_ptr(), stream)
        assert rc == 0, rbc.load().rbc_last_error().decode()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ref_ids.cpu().numpy())
        a = dist.cpu().numpy().astype(np.float64)
        b = ref_dist.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(a - b) <= DIST_REL * np.maximum(b, 1e-30))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    f = _entry()
    X = torch.zeros((64, 8), device="cuda")
    m = 200_000  # more query tiles than the 32 MiB scratch holds at k = 10
    Q = torch.zeros((m, 8), device="cuda")
    ids = torch.empty((m, 10), dtype=torch.int64, device="cuda")
    dist = torch.empty((m, 10), dtype=torch.float32, device="cuda")
    rc = f(Q.data_ptr(), m, X.data_ptr(), 64, 8, 10, rbc.L2, ids.data_ptr(), dist.data_ptr(), None)
    assert rc == -5
    assert "scratch" in rbc.load().rbc_last_error().decode()


def test_noalloc_rejects_host_buffers():
    f = _entry()
    X = np.zeros((64, 8), np.float32)
    Q = np.zeros((4, 8), np.float32)
    ids = np.empty((4, 2), np.int64)
    dist = np.empty((4, 2), np.float32)
    rc = f(Q.ctypes.data, 4, X.ctypes.data, 64, 8, 2, rbc.L2, ids.ctypes.data, dist.ctypes.data, None)
    assert rc == -1

"""rbc_search recorded in a CUDA graph and replayed (windowed plan).

The windowed exact search (Section 5.2 with sorted lists) takes every
overflow decision on the device, so a call made while the stream is captured
reads nothing back: the graph holds the whole search, and each replay on new
query values must give the exact k nearest neighbours, element by element
against the FP64 oracle's brute force (Section 3)."""
import numpy as np
import pytest

import oracle
import synth
from parity import check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

MET = {"l2": rbc.L2, "l1": rbc.L1}


def record(idx, Qs, k):
    """Static outputs, one eager call (kernel attributes, pinned statistics
    block), then the same call recorded into a graph."""
    ids = torch.empty((Qs.shape[0], k), dtype=torch.int64, device="cuda")
    dist = torch.empty((Qs.shape[0], k), dtype=torch.float32, device="cuda")
    rbc.rbc_search(idx, Qs, k, out_ids=ids, out_dist=dist)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        rbc.rbc_search(idx, Qs, k, out_ids=ids, out_dist=dist)
    torch.cuda.synchronize()
    return g, ids, dist


@pytest.mark.parametrize(
    "storage,metric,plan",
    [(rbc.BF16, "l2", rbc.PLAN_WINDOW), (rbc.F32, "l2", rbc.PLAN_WINDOW),
     (rbc.F32, "l1", rbc.PLAN_WINDOW)],
)
def test_replays_match_oracle(storage, metric, plan):
    X, _ = synth.make_workload("iid-n16k-d16", seed=0)
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), 128, metric=MET[metric], seed=2,
                        storage=storage, plan=plan)
    m, k = 700, 10  # several 128-query chunks and a ragged tail
    Qs = torch.empty((m, X.shape[1]), dtype=torch.float32, device="cuda")
    Qs.copy_(torch.from_numpy(synth.iid_normal(m, X.shape[1], 11)))
    g, ids, dist = record(idx, Qs, k)
    for seed in (21, 22, 23):
        Q = synth.iid_normal(m, X.shape[1], seed)
        Qs.copy_(torch.from_numpy(Q))
        ids.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        o_ids, o_rho = oracle.bf(Q, X, k, metric)
        check_knn(Q, X, ids.cpu().numpy(), dist.cpu().numpy(), o_ids, o_rho, metric)
    rbc.search_check(idx)
    # the eager call on the last queries agrees with the replay
    e_ids, e_dist = rbc.rbc_search(idx, Qs, k)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(e_ids.cpu().numpy(), ids.cpu().numpy())
    np.testing.assert_array_equal(e_dist.cpu().numpy(), dist.cpu().numpy())
    idx.close()


def test_replay_finishes_rows_that_overflow_twice():
    # 9000 copies of one point: more candidates than a query's buffer holds
    # (8192) even after the re-threshold, so inside the graph these rows are
    # finished by the FP64 band pass; the ties go to the smallest ids
    X = synth.iid_normal(30000, 24, 3)
    X[5000:14000] = X[5000]
    Q = np.concatenate([X[5000:5001].repeat(3, 0), synth.iid_normal(300, 24, 4)]).astype(np.float32)
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), 170, seed=6, storage=rbc.BF16)
    Qs = torch.from_numpy(Q).cuda()
    g, ids, dist = record(idx, Qs, 10)
    ids.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    got_ids, got_dist = ids.cpu().numpy(), dist.cpu().numpy()
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    check_knn(Q, X, got_ids, got_dist, o_ids, o_rho)
    np.testing.assert_array_equal(got_ids[:3], np.tile(np.arange(5000, 5010), (3, 1)))
    rbc.search_check(idx)
    idx.close()


@pytest.mark.parametrize("plan", [rbc.PLAN_TILE_UNION, rbc.PLAN_WINDOW_OFFSET])
def test_capture_rejects_other_plans_and_host_memory(plan):
    # the tile-union plan and the offset plan read counts back mid-search
    X, Q = synth.make_workload("iid-n16k-d16", seed=0)
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), 128, seed=2, storage=rbc.BF16, plan=plan)
    Qs = torch.from_numpy(Q[:256]).cuda()
    ids = torch.empty((256, 5), dtype=torch.int64, device="cuda")
    dist = torch.empty((256, 5), dtype=torch.float32, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with pytest.raises(rbc.RbcError):
        with torch.cuda.graph(g, stream=s):
            rbc.rbc_search(idx, Qs, 5, out_ids=ids, out_dist=dist)
    idx.close()
    torch.cuda.synchronize()

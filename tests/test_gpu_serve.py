"""The serving engine on the GPU: requests of mixed sizes merged into batches
give the same neighbours as each request searched alone (ids exact outside
near-ties of 1e-6 relative, distances within 1e-5 relative) and as the FP64
oracle; batches of different workers overlap on the device; admission keeps
the in-flight workspace bounds within the HBM budget; and the workspace bound
of rbc_search holds for every plan."""
import numpy as np
import pytest

import oracle
import synth
from parity import DIST_REL, TIE_REL, check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

N, D, N_R = 200_000, 96, 448


@pytest.fixture(scope="module")
def served():
    w = synth.WORKLOADS["sincos12-n8m-d96"]
    X, Q = synth.make_workload(w, seed=0, n=N, m=40_000)
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), N_R, seed=2, storage=rbc.F16)
    torch.cuda.synchronize()
    yield X, Q, idx
    idx.close()


def requests(rng, Q, count, lo=1, hi=4096, ks=(1, 5, 10)):
    """(start, m, k) of requests with log-uniform sizes over rows of Q."""
    out = []
    for _ in range(count):
        m = int(np.exp(rng.uniform(np.log(lo), np.log(hi + 1))))
        m = max(lo, min(hi, m))
        s = int(rng.integers(0, len(Q) - m + 1))
        out.append((s, m, int(rng.choice(ks))))
    return out


def alone(idx, Q, k):
    ids, dist = rbc.rbc_search(idx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), k)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def assert_same(ids, dist, ids_a, dist_a):
    """Same result within the parity tolerance: ids may differ only where the
    two runs' distances at that rank form a near-tie."""
    np.testing.assert_allclose(dist, dist_a, rtol=DIST_REL, atol=0)
    diff = ids != ids_a
    if diff.any():
        da, db = dist[diff].astype(np.float64), dist_a[diff].astype(np.float64)
        assert np.all(np.abs(da - db) <= TIE_REL * np.maximum(db, 1e-30)), "ids differ outside a tie"


def test_mix_equals_alone_and_oracle(served):
    X, Q, idx = served
    rng = np.random.default_rng(7)
    reqs = requests(rng, Q, 48)
    with rbc.Server(idx, workers=3, max_batch=8192, k_max=10) as srv:
        tickets = [srv.submit(Q[s : s + m], k) for s, m, k in reqs]
        out = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["requests"] == len(reqs) and st["queries"] == sum(m for _, m, _ in reqs)
    # arrivals were merged: some batch served several requests
    assert max(info["batch_requests"] for _, _, info in out) > 1
    assert st["batches"] < len(reqs)
    for (s, m, k), (ids, dist, info) in zip(reqs, out):
        assert info["status"] == 0 and ids.shape == (m, k)
        assert info["t_submit_ns"] <= info["t_start_ns"] <= info["t_done_ns"]
        ids_a, dist_a = alone(idx, Q[s : s + m], k)
        assert_same(ids, dist, ids_a, dist_a)
    # the FP64 oracle on a sample of every request's rows
    for (s, m, k), (ids, dist, _) in list(zip(reqs, out))[::4]:
        rows = np.unique(np.linspace(0, m - 1, min(m, 24)).astype(int))
        o_ids, o_rho = oracle.bf(Q[s + rows], X, k)
        check_knn(Q[s + rows], X, ids[rows], dist[rows], o_ids, o_rho)


def test_batches_overlap_on_the_device(served):
    _, Q, idx = served
    with rbc.Server(idx, workers=2, max_batch=4096, k_max=10) as srv:
        tickets = [srv.submit(Q[i * 4096 : (i + 1) * 4096], 10) for i in range(8)]
        infos = [srv.wait(t)[2] for t in tickets]
        st = srv.stats()
    assert st["max_in_flight"] == 2
    spans = sorted({(i["t_start_ns"], i["t_done_ns"]) for i in infos})
    assert any(a[1] > b[0] for a, b in zip(spans, spans[1:])), "no two batches ran at the same time"


def test_admission_keeps_reserved_workspace_within_budget(served):
    _, Q, idx = served
    one = rbc.search_workspace(idx, 4096, 10)
    budget = int(one * 1.5)  # room for one full batch at a time
    rng = np.random.default_rng(3)
    reqs = requests(rng, Q, 24, lo=256, hi=4096, ks=(10,))
    with rbc.Server(idx, workers=3, max_batch=16384, k_max=10, hbm_budget=budget) as srv:
        tickets = [srv.submit(Q[s : s + m], k) for s, m, k in reqs]
        out = [srv.wait(t) for t in tickets]
        st = srv.stats()
        # a request whose batch alone could never fit the budget is refused
        big = np.ascontiguousarray(Q[:16384])
        if rbc.search_workspace(idx, 16384, 10) > budget:
            with pytest.raises(rbc.RbcError) as e:
                srv.submit(big, 10)
            assert e.value.code == -2
    assert st["peak_reserved_bytes"] <= budget
    for _, _, info in out:
        assert rbc.search_workspace(idx, info["batch_queries"], 10) <= budget
    for (s, m, k), (ids, dist, _) in zip(reqs[::3], out[::3]):
        ids_a, dist_a = alone(idx, Q[s : s + m], k)
        assert_same(ids, dist, ids_a, dist_a)


def test_request_validation_and_empty_request(served):
    _, Q, idx = served
    with rbc.Server(idx, workers=1, max_batch=1024, k_max=5) as srv:
        for kw in [dict(Q=Q[:10], k=6), dict(Q=Q[:1025], k=1), dict(Q=Q[:10], k=0)]:
            with pytest.raises(rbc.RbcError) as e:
                srv.submit(kw["Q"], kw["k"])
            assert e.value.code == -1
        t = srv.submit(np.zeros((0, D), np.float32), 3)
        ids, dist, info = srv.wait(t)
        assert ids.shape == (0, 3) and info["batch"] == -1 and info["status"] == 0
        with pytest.raises(rbc.RbcError):
            srv.wait(t)  # collected already
        t = srv.submit(Q[:7], 5)
        ids, dist, _ = srv.wait(t, timeout_us=30_000_000)
        ids_a, dist_a = alone(idx, Q[:7], 5)
        assert_same(ids, dist, ids_a, dist_a)


@pytest.mark.parametrize(
    "gen,storage,metric,mode,plan",
    [
        ("subspace", rbc.BF16, rbc.L2, rbc.EXACT, rbc.PLAN_WINDOW),
        ("subspace", rbc.BF16, rbc.L2, rbc.EXACT, rbc.PLAN_TILE_UNION),
        ("subspace", rbc.BF16, rbc.L2, rbc.EXACT, rbc.PLAN_WINDOW_OFFSET),
        ("subspace", rbc.F32, rbc.L2, rbc.EXACT, rbc.PLAN_WINDOW),
        ("subspace", rbc.F32, rbc.L1, rbc.EXACT, rbc.PLAN_WINDOW),
        ("subspace", rbc.BF16, rbc.L2, rbc.ONESHOT, rbc.PLAN_WINDOW),
        ("subspace", rbc.F32, rbc.L2, rbc.ONESHOT, rbc.PLAN_WINDOW),
        ("subspace", rbc.FP8E4M3, rbc.L2, rbc.EXACT, rbc.PLAN_WINDOW),
        ("subspace", rbc.FP8E4M3, rbc.L2, rbc.ONESHOT, rbc.PLAN_WINDOW),
    ],
)
def test_workspace_bound_holds(gen, storage, metric, mode, plan):
    X, Q = synth.make_workload("subspace8-n1m-d64", seed=0, n=60_000, m=9000)
    kw = dict(s=256) if mode == rbc.ONESHOT else {}
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), 245, metric=metric, seed=2, storage=storage,
                        mode=mode, plan=plan, **kw)
    Qd = torch.from_numpy(Q).cuda()
    for m in (1, 130, 3000, 9000):
        for k in (1, 10):
            rbc.rbc_search(idx, Qd[:m], k)
            got = rbc.last_stats()["workspace_bytes"]
            bound = rbc.search_workspace(idx, m, k)
            assert 0 < got <= bound, (m, k, got, bound)
    # host inputs and outputs: the I/O copies are part of the workspace
    rbc.rbc_search(idx, Q[:500], 10)
    got = rbc.last_stats()["workspace_bytes"]
    assert got <= rbc.search_workspace(idx, 500, 10)
    idx.close()

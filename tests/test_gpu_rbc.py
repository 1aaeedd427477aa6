"""Parity of the CUDA Random Ball Cover with the FP64 oracle (Sections 4-5):
the build (representatives, lists, radii) against the oracle's build, and the
exact search against the oracle's brute force (the exact algorithm returns
exactly the brute-force neighbours)."""
import numpy as np
import pytest

import oracle
import synth
from parity import check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

MET = {"l2": rbc.L2, "l1": rbc.L1}


def build(X, n_r, metric="l2", seed=2, storage=rbc.F32, **kw):
    return rbc.rbc_build(torch.from_numpy(X).cuda(), n_r, metric=MET[metric], seed=seed, storage=storage, **kw)


def search(idx, Q, k):
    ids, dist = rbc.rbc_search(idx, torch.from_numpy(Q).cuda(), k)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_build_matches_oracle(metric):
    X, _ = synth.make_workload("iid-n16k-d16", seed=0)
    idx = build(X, 128, metric)
    ex = idx.export()
    reps = oracle.sample_reps(len(X), 128, 2)
    np.testing.assert_array_equal(ex["reps"], reps)
    o = oracle.build_exact(X, reps, metric)
    sizes = np.array([len(l) for l in o.lists])
    np.testing.assert_array_equal(np.diff(ex["offsets"]), sizes)
    for r in range(128):
        got = ex["members"][ex["offsets"][r] : ex["offsets"][r + 1]]
        np.testing.assert_array_equal(np.sort(got), o.lists[r])
        # each list is ordered by distance to its representative (FP32 values,
        # so FP64 distances may step back only within rounding), then by id
        dg = oracle.dist(X[reps[r] : reps[r] + 1], X[got], metric)[0]
        assert np.all(np.diff(dg) >= -1e-5 * dg[1:]), r
    # radii: an upper bound within the FP32 rounding allowance
    assert np.all(ex["psi"] >= o.psi * (1 - 1e-6))
    assert np.all(ex["psi"] <= o.psi * (1 + 2e-5) + 1e-6)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("k", [1, 10])
def test_exact_search_iid_n16k_d16(metric, k):
    X, Q = synth.make_workload("iid-n16k-d16", seed=0)
    idx = build(X, 128, metric)
    ids, dist = search(idx, Q, k)
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)
    st = rbc.last_stats()
    assert st["queries"] == len(Q) and st["kept_reps"] >= len(Q)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("n,m,d,n_r,k", [(5000, 300, 5, 71, 3), (2049, 129, 33, 1, 2), (3001, 77, 12, 3001, 4), (20000, 513, 8, 141, 7), (1000, 1, 64, 30, 31)])
@pytest.mark.parametrize("plan", [rbc.PLAN_WINDOW, rbc.PLAN_TILE_UNION])
def test_exact_search_ragged(metric, n, m, d, n_r, k, plan):
    # FP32 storage: both stage-two plans on the CUDA cores
    X = synth.iid_normal(n, d, 10 + n)
    Q = synth.iid_normal(m, d, 20 + m)
    idx = build(X, n_r, metric, seed=n_r, plan=plan)
    ids, dist = search(idx, Q, k)
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("k", [1, 10])
def test_exact_search_f32_window_subspace(metric, k):
    # the windowed plan on the CUDA cores examines fewer (query, point) pairs
    # than the tile-union plan and returns the same neighbours
    X, Q = synth.make_workload("subspace8-n1m-d64", seed=0, n=60000, m=700)
    res = {}
    for plan in (rbc.PLAN_WINDOW, rbc.PLAN_TILE_UNION):
        idx = build(X, 245, metric, plan=plan)
        res[plan] = search(idx, Q, k) + (rbc.last_stats(),)
        idx.close()
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    for plan, (ids, dist, st) in res.items():
        check_knn(Q, X, ids, dist, o_ids, o_rho, metric)
    assert res[rbc.PLAN_WINDOW][2]["pairs"] < res[rbc.PLAN_TILE_UNION][2]["pairs"]


def test_exact_search_subspace_workload_small():
    mod = synth.SubspaceModel(d=64, k=8, noise_var=0.01, seed=0)
    X = mod.sample(60000, 0)
    Q = mod.sample(700, 1)
    idx = build(X, 245)
    for k in (1, 10):
        ids, dist = search(idx, Q, k)
        o_ids, o_rho = oracle.bf(Q, X, k, "l2")
        check_knn(Q, X, ids, dist, o_ids, o_rho)


def test_exact_search_with_duplicates():
    base = synth.iid_normal(60, 4, 30)
    X = np.concatenate([base, base, base[:25], base[:5]])
    Q = np.concatenate([base[:15], synth.iid_normal(40, 4, 31)])
    for n_r in (1, 9, 60, len(X)):
        idx = build(X, n_r, seed=n_r)
        ids, dist = search(idx, Q, 5)
        o_ids, o_rho = oracle.bf(Q, X, 5, "l2")
        np.testing.assert_array_equal(ids, o_ids)


def test_given_representatives():
    X = synth.iid_normal(3000, 6, 40)
    Q = synth.iid_normal(100, 6, 41)
    reps = np.arange(0, 3000, 37)
    idx = build(X, len(reps), rep_ids=reps)
    np.testing.assert_array_equal(idx.export()["reps"], reps)
    ids, dist = search(idx, Q, 3)
    o_ids, o_rho = oracle.bf(Q, X, 3, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)


def test_host_buffer_search():
    X = synth.iid_normal(4000, 10, 50)
    Q = synth.iid_normal(200, 10, 51)
    idx = rbc.rbc_build(X, 63, seed=3)  # numpy database
    ids, dist = rbc.rbc_search(idx, Q, 4)  # numpy queries and outputs
    o_ids, o_rho = oracle.bf(Q, X, 4, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)


@pytest.mark.parametrize("storage,plan", [(rbc.F32, rbc.PLAN_WINDOW), (rbc.BF16, rbc.PLAN_WINDOW),
                                          (rbc.BF16, rbc.PLAN_WINDOW_OFFSET)])
@pytest.mark.parametrize("pinned,own_stream", [(False, False), (True, False), (True, True)])
def test_host_rows_copied_beside_stage_one(storage, plan, pinned, own_stream):
    # n_r = 4096 cuts 74,537 queries into batches of 65,536 and 9,001 rows;
    # each copies its host rows in eight chunks on a second stream, and each
    # chunk's per-row steps (stage 1, row statistics, low-precision rows)
    # wait for its own copy only (the second batch: chunks of 1,152 rows and
    # a ragged last one of 937).  test_host_buffer_search covers a batch
    # below the chunking threshold (one copy).  The answers must equal those
    # of the same search on device buffers.
    X = synth.iid_normal(40000, 32, 70)
    Q = synth.iid_normal(74537, 32, 71)
    k = 5
    idx = build(X, 4096, storage=storage, plan=plan)
    dev_ids, dev_dist = search(idx, Q, k)
    Qh = torch.from_numpy(Q)
    ids = torch.empty((Q.shape[0], k), dtype=torch.int64)
    dist = torch.empty((Q.shape[0], k), dtype=torch.float32)
    if pinned:
        Qh, ids, dist = Qh.pin_memory(), ids.pin_memory(), dist.pin_memory()
    # own_stream: the search runs on a stream of its own (not the legacy
    # default stream), which the copy stream's events must order against
    rbc.rbc_search(idx, Qh, k, out_ids=ids, out_dist=dist,
                   stream=torch.cuda.Stream() if own_stream else None)
    np.testing.assert_array_equal(ids.numpy(), dev_ids)
    np.testing.assert_array_equal(dist.numpy(), dev_dist)
    sample = np.random.default_rng(72).choice(Q.shape[0], 300, replace=False)
    sample[:2] = [0, Q.shape[0] - 1]
    o_ids, o_rho = oracle.bf(Q[sample], X, k, "l2")
    check_knn(Q[sample], X, ids.numpy()[sample], dist.numpy()[sample], o_ids, o_rho)


def test_empty_query_batch():
    X = synth.iid_normal(500, 4, 60)
    idx = build(X, 22)
    ids, dist = search(idx, np.zeros((0, 4), np.float32), 2)
    assert ids.shape == (0, 2)


# ---- low-precision storage: tensor-core stage two (windowed emission or
# tile-union top-c lists), exact re-rank ----

PLANS = [rbc.PLAN_WINDOW, rbc.PLAN_TILE_UNION, rbc.PLAN_WINDOW_OFFSET]
WINDOW_PLANS = [rbc.PLAN_WINDOW, rbc.PLAN_WINDOW_OFFSET]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("storage", [rbc.BF16, rbc.F16, rbc.FP8E4M3])
@pytest.mark.parametrize("k", [1, 10])
def test_exact_search_tc_iid_n16k_d16(storage, k, plan):
    X, Q = synth.make_workload("iid-n16k-d16", seed=0)
    idx = build(X, 128, storage=storage, plan=plan)
    ids, dist = search(idx, Q, k)
    o_ids, o_rho = oracle.bf(Q, X, k, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("n,m,d,n_r,k", [(5000, 300, 5, 71, 3), (2049, 129, 33, 1, 2), (3001, 77, 12, 3001, 4), (20000, 513, 100, 141, 7), (1000, 1, 64, 30, 31), (40, 20, 8, 3, 31), (9000, 700, 250, 90, 10)])
def test_exact_search_tc_ragged(n, m, d, n_r, k, plan):
    X = synth.iid_normal(n, d, 10 + n)
    Q = synth.iid_normal(m, d, 20 + m)
    idx = build(X, n_r, seed=n_r, storage=rbc.BF16, plan=plan)
    ids, dist = search(idx, Q, k)
    o_ids, o_rho = oracle.bf(Q, X, k, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)


@pytest.mark.parametrize("n,m,d,n_r,k", [(5000, 300, 5, 71, 3), (3001, 77, 12, 3001, 4), (20000, 513, 100, 141, 7), (1000, 1, 64, 30, 31), (9000, 700, 250, 90, 10)])
def test_exact_search_fp8_ragged(n, m, d, n_r, k):
    # FP8 storage always takes the tile-union plan (per-column scales)
    X = synth.iid_normal(n, d, 10 + n)
    Q = synth.iid_normal(m, d, 20 + m)
    idx = build(X, n_r, seed=n_r, storage=rbc.FP8E4M3)
    ids, dist = search(idx, Q, k)
    o_ids, o_rho = oracle.bf(Q, X, k, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)
    assert idx.info()["storage"] == rbc.FP8E4M3


@pytest.mark.parametrize("plan", PLANS)
def test_exact_search_tc_subspace_workload_small(plan):
    mod = synth.SubspaceModel(d=64, k=8, noise_var=0.01, seed=0)
    X = mod.sample(60000, 0)
    Q = mod.sample(700, 1)
    idx = build(X, 245, storage=rbc.BF16, plan=plan)
    for k in (1, 10):
        ids, dist = search(idx, Q, k)
        o_ids, o_rho = oracle.bf(Q, X, k, "l2")
        check_knn(Q, X, ids, dist, o_ids, o_rho)


@pytest.mark.parametrize("plan", PLANS)
def test_exact_search_tc_duplicates(plan):
    base = synth.iid_normal(60, 4, 30)
    X = np.concatenate([base, base, base[:25], base[:5]])
    Q = np.concatenate([base[:15], synth.iid_normal(40, 4, 31)])
    for n_r in (1, 9, 60, len(X)):
        idx = build(X, n_r, seed=n_r, storage=rbc.BF16, plan=plan)
        ids, dist = search(idx, Q, 5)
        o_ids, o_rho = oracle.bf(Q, X, 5, "l2")
        np.testing.assert_array_equal(ids, o_ids)


@pytest.mark.parametrize("plan", PLANS)
def test_exact_search_multi_batch_with_recheck(plan):
    """More queries than one internal batch (131,072), with 40 exact copies of
    some points so that queries sitting on them tie far past the candidate
    width: the tile-union plan fails the low-precision certificate and
    re-searches them (every batch must re-search its own rows only); the
    windowed plan takes every copy as a candidate and settles the order in
    FP64."""
    base = synth.iid_normal(2000, 16, 90)
    X = np.concatenate([base] + [base[:100]] * 40)
    g = np.random.default_rng(91)
    m = 140_000
    Q = (X[g.integers(0, len(X), m)] + g.normal(0, 0.05, (m, 16))).astype(np.float32)
    on = np.arange(0, m, 50)
    Q[on] = base[g.integers(0, 100, len(on))]  # exactly on a 41-fold point
    idx = build(X, 80, storage=rbc.BF16, plan=plan)
    ids, dist = search(idx, Q, 5)
    st = rbc.last_stats()
    if plan == rbc.PLAN_TILE_UNION:
        assert st["uncertified"] > 0  # the recheck path ran
    else:
        assert st["fp64_ties"] > 0
    ref_ids, ref_dist = rbc.bf_search(torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda(), 5)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ids, ref_ids.cpu().numpy())
    sel = np.unique(np.concatenate([on[:300], g.choice(m, 1200, replace=False)]))
    o_ids, o_rho = oracle.bf(Q[sel], X, 5, "l2")
    check_knn(Q[sel], X, ids[sel], dist[sel], o_ids, o_rho)
    np.testing.assert_array_equal(ids[on[:300]], o_ids[np.searchsorted(sel, on[:300])])


@pytest.mark.parametrize("storage,metric", [(rbc.BF16, "l2"), (rbc.F32, "l2"), (rbc.F32, "l1")])
@pytest.mark.parametrize("k", [1, 10, 20])
def test_exact_search_fewer_queries_than_lists(storage, metric, k):
    # m <= n_r: most lists hold one query or none, so the own-list tiles are
    # almost all padding rows
    X, _ = synth.make_workload("iid-n16k-d16", seed=0)
    Q = synth.iid_normal(300, 16, 17)
    idx = build(X, 512, metric, storage=storage)
    ids, dist = search(idx, Q, k)
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("plan", WINDOW_PLANS)
def test_window_many_tied_candidates_are_streamed(plan):
    # 700 copies of one point: a query on it has 700 survivors at distance 0,
    # more than the shared-memory re-rank holds; they are re-ranked in a
    # stream (no FP32 re-search) and the ties go to the smallest ids
    X = synth.iid_normal(20000, 24, 3)
    X[5000:5700] = X[5000]
    Q = np.concatenate([X[5000:5001].repeat(3, 0), synth.iid_normal(300, 24, 4)]).astype(np.float32)
    idx = build(X, 140, storage=rbc.BF16, seed=6, plan=plan)
    ids, dist = search(idx, Q, 10)
    assert rbc.last_stats()["uncertified"] == 0
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)
    np.testing.assert_array_equal(ids[:3], np.tile(np.arange(5000, 5010), (3, 1)))


@pytest.mark.parametrize("plan", WINDOW_PLANS)
def test_window_candidate_overflow_goes_to_fp32_research(plan):
    # 9000 copies of one point: more candidates than a query's buffer holds
    # (8192), so those queries are searched again in FP32 (the offset plan's
    # stored estimates bound the re-threshold of the dense pass)
    X = synth.iid_normal(30000, 24, 3)
    X[5000:14000] = X[5000]
    Q = np.concatenate([X[5000:5001].repeat(3, 0), synth.iid_normal(300, 24, 4)]).astype(np.float32)
    idx = build(X, 170, storage=rbc.BF16, seed=6, plan=plan)
    ids, dist = search(idx, Q, 10)
    assert rbc.last_stats()["uncertified"] >= 3
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)
    np.testing.assert_array_equal(ids[:3], np.tile(np.arange(5000, 5010), (3, 1)))


@pytest.mark.parametrize("plan", WINDOW_PLANS)
def test_searches_after_an_arena_overflow_agree(plan):
    # the 9000 copies overflow the emission's hit arena: the hits past a full
    # slice go to the query buffers directly, and every search gives the
    # same answer
    X = synth.iid_normal(30000, 24, 3)
    X[5000:14000] = X[5000]
    Q = np.concatenate([X[5000:5001].repeat(3, 0), synth.iid_normal(300, 24, 4)]).astype(np.float32)
    idx = build(X, 170, storage=rbc.BF16, seed=6, plan=plan)
    ids0, dist0 = search(idx, Q, 10)
    for _ in range(12):
        ids, dist = search(idx, Q, 10)
        np.testing.assert_array_equal(ids, ids0)
        np.testing.assert_array_equal(dist, dist0)
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    check_knn(Q, X, ids0, dist0, o_ids, o_rho)
    Q2 = synth.iid_normal(500, 24, 5)
    ids2, dist2 = search(idx, Q2, 5)
    o_ids, o_rho = oracle.bf(Q2, X, 5, "l2")
    check_knn(Q2, X, ids2, dist2, o_ids, o_rho)


def test_window_stats_count_fewer_pairs_than_tile_union():
    mod = synth.SubspaceModel(d=64, k=8, noise_var=0.01, seed=0)
    X = mod.sample(120000, 0)
    Q = mod.sample(4000, 1)
    res = {}
    for plan in PLANS:
        idx = build(X, 350, storage=rbc.BF16, plan=plan)
        ids, dist = search(idx, Q, 10)
        res[plan] = (ids, rbc.last_stats())
    np.testing.assert_array_equal(res[rbc.PLAN_WINDOW][0], res[rbc.PLAN_TILE_UNION][0])
    assert res[rbc.PLAN_WINDOW][1]["pairs"] < res[rbc.PLAN_TILE_UNION][1]["pairs"]


@pytest.mark.parametrize("d", [64, 96, 128])
def test_offset_plan_on_tight_clusters(d):
    """Thirty Gaussian clusters, centres N(0, I), sigma in [0.05, 0.5], two
    representatives per cluster: the bf16 rounding of x grows with |x| (about
    sqrt(d)), that of x - r with the cluster's size, so the offset plan emits
    fewer candidates than the plain windowed plan; both answers match the
    oracle (d = 96: the norm pair rides in the rows' padding)."""
    mod = synth.ClusterModel(d=d, n_clusters=30, seed=0)
    X, Q = mod.sample(60000, 0), mod.sample(600, 1)
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    cands = {}
    for plan in WINDOW_PLANS:
        idx = build(X, 60, storage=rbc.BF16, seed=3, plan=plan)
        ids, dist = search(idx, Q, 10)
        cands[plan] = rbc.last_stats()["candidates"]
        check_knn(Q, X, ids, dist, o_ids, o_rho)
        idx.close()
    assert cands[rbc.PLAN_WINDOW_OFFSET] < cands[rbc.PLAN_WINDOW], cands


@pytest.mark.parametrize("n_r", [1, 3, 4000])
def test_offset_plan_edge_lists(n_r):
    """Offsets from the representative when one list holds everything (n_r =
    1), a few long lists, and lists of one point each (every row y = 0 and
    the query rows a = q - r carry the whole distance); queries that are
    database points (distance 0) and far ones."""
    X = synth.iid_normal(4000, 16, 40)
    Q = np.concatenate([X[:50], synth.iid_normal(200, 16, 41), 30.0 * synth.iid_normal(20, 16, 42)])
    Q = Q.astype(np.float32)
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    idx = build(X, n_r, storage=rbc.BF16, seed=5, plan=rbc.PLAN_WINDOW_OFFSET)
    ids, dist = search(idx, Q, 10)
    check_knn(Q, X, ids, dist, o_ids, o_rho)
    idx.close()

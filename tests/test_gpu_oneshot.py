"""Parity of the CUDA one-shot Random Ball Cover with the FP64 oracle
(Sections 4 and 5.1): the build (each list L_r = the s nearest points of r in
(rho, id) order, psi_r = the s-th distance) and the search (nearest
representative, then brute force over its list) against the oracle's
one-shot build and search on the same representatives."""
import numpy as np
import pytest

import oracle
import synth
from parity import TIE_REL, check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

MET = {"l2": rbc.L2, "l1": rbc.L1}


def build(X, n_r, s, metric="l2", seed=2, storage=rbc.F32, **kw):
    return rbc.rbc_build(torch.from_numpy(X).cuda(), n_r, metric=MET[metric], seed=seed,
                         mode=rbc.ONESHOT, s=s, storage=storage, **kw)


def search(idx, Q, k):
    ids, dist = rbc.rbc_search(idx, torch.from_numpy(Q).cuda(), k)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def check_lists(X, reps, members, s, o_lists, metric):
    """Every list equals the oracle's, except that entries may trade places
    among points whose FP64 distances to r agree within the tie tolerance."""
    got = members.reshape(len(reps), s)
    diff = 0
    for r in range(len(reps)):
        g, o = got[r], o_lists[r]
        if np.array_equal(g, o):
            continue
        diff += 1
        assert len(set(g.tolist())) == s, f"list {r} holds duplicate ids"
        rr = X[reps[r] : reps[r] + 1]
        dg = oracle.dist(rr, X[g], metric)[0]
        do = oracle.dist(rr, X[o], metric)[0]
        np.testing.assert_allclose(dg, do, rtol=TIE_REL, atol=1e-30, err_msg=f"list {r}")
    return diff


def check_search(X, Q, o_index, ids, dist, k, metric):
    """Search results equal the oracle's one-shot answer.  Where the nearest
    representative itself is a near-tie, either tied representative's list is
    a correct answer."""
    o_ids, o_rho, near = oracle.search_oneshot(o_index, Q, k)
    R = X[o_index.reps]
    Dr = oracle.dist(Q, R, metric)
    srt = np.sort(Dr, axis=1)
    amb = np.zeros(len(Q), dtype=bool)
    if Dr.shape[1] > 1:
        amb = srt[:, 1] - srt[:, 0] <= TIE_REL * np.maximum(srt[:, 0], 1e-30)
    ok = ~amb
    if ok.any():
        check_knn(Q[ok], X, ids[ok], dist[ok], o_ids[ok], o_rho[ok], metric)
    for i in np.nonzero(amb)[0]:
        cands = np.nonzero(Dr[i] <= srt[i, 0] * (1 + TIE_REL) + 1e-30)[0]
        passed = False
        for r in cands:
            a_ids, a_rho = oracle.bf_lists(Q[i : i + 1], X, [o_index.lists[r]], k, metric)
            try:
                check_knn(Q[i : i + 1], X, ids[i : i + 1], dist[i : i + 1], a_ids, a_rho, metric)
                passed = True
                break
            except AssertionError:
                pass
        assert passed, f"query {i}: result matches no tied representative's list"


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_oneshot_build_matches_oracle(metric):
    X, _ = synth.make_workload("iid-n16k-d16", seed=0)
    s = 128
    idx = build(X, 128, s, metric)
    info = idx.info()
    assert info["mode"] == rbc.ONESHOT and info["s"] == s and info["list_entries"] == 128 * s
    ex = idx.export()
    reps = oracle.sample_reps(len(X), 128, 2)
    np.testing.assert_array_equal(ex["reps"], reps)
    np.testing.assert_array_equal(ex["offsets"], np.arange(129) * s)
    o = oracle.build_oneshot(X, reps, s, metric)
    check_lists(X, reps, ex["members"], s, o.lists, metric)
    np.testing.assert_allclose(ex["psi"], o.psi, rtol=1e-6)
    # r is its own nearest point (rho(r, r) = 0)
    assert np.all(ex["members"].reshape(128, s)[:, 0] == reps)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("k", [1, 10])
def test_oneshot_search_iid_n16k_d16(metric, k):
    X, Q = synth.make_workload("iid-n16k-d16", seed=0)
    n_r, s = 128, 256
    idx = build(X, n_r, s, metric)
    ids, dist = search(idx, Q, k)
    o = oracle.build_oneshot(X, oracle.sample_reps(len(X), n_r, 2), s, metric)
    check_search(X, Q, o, ids, dist, k, metric)
    st = rbc.last_stats()
    assert st["queries"] == len(Q) and st["kept_reps"] == len(Q)
    assert st["pairs"] == len(Q) * s
    assert st["tile_points"] * 128 >= st["pairs"]  # tiles of at most 128 queries


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize(
    "n,m,d,n_r,s,k",
    [
        (5000, 300, 5, 71, 50, 3),
        (2049, 129, 33, 1, 2049, 2),  # one list holding every point: brute force
        (3001, 77, 12, 3001, 1, 1),  # every point a representative, lists of one
        (20000, 513, 8, 141, 300, 7),
        (1000, 1, 64, 30, 31, 31),  # k = s
        (4099, 1000, 3, 5, 700, 5),  # few representatives: many tiles per list
    ],
)
def test_oneshot_search_ragged(metric, n, m, d, n_r, s, k):
    X = synth.iid_normal(n, d, 10 + n)
    Q = synth.iid_normal(m, d, 20 + m)
    idx = build(X, n_r, s, metric, seed=n_r)
    o = oracle.build_oneshot(X, oracle.sample_reps(n, n_r, n_r), s, metric)
    ex = idx.export()
    check_lists(X, o.reps, ex["members"], s, o.lists, metric)
    ids, dist = search(idx, Q, k)
    check_search(X, Q, o, ids, dist, k, metric)


def test_oneshot_queries_clustered_on_few_representatives():
    # 900 queries near three representatives: several padded tiles per list,
    # most representatives without queries
    X = synth.iid_normal(30000, 16, 5)
    n_r, s = 200, 400
    idx = build(X, n_r, s, seed=9)
    reps = oracle.sample_reps(len(X), n_r, 9)
    rng = np.random.default_rng(3)
    Q = np.concatenate([X[reps[j]] + 0.05 * rng.standard_normal((300, 16)) for j in (0, 7, 150)])
    Q = Q.astype(np.float32)
    ids, dist = search(idx, Q, 8)
    o = oracle.build_oneshot(X, reps, s)
    check_search(X, Q, o, ids, dist, 8, "l2")


def test_oneshot_duplicates_exceed_candidate_capacity():
    # 300 copies of one point at a representative: 300 points tie at distance
    # zero for a list of s = 64, more than the first candidate capacity
    X = synth.iid_normal(8000, 8, 1)
    X[1000:1300] = X[1000]
    reps = np.array(sorted({1000, *range(0, 8000, 97)}), dtype=np.int64)
    s = 64
    idx = rbc.rbc_build(torch.from_numpy(X).cuda(), len(reps), mode=rbc.ONESHOT, s=s,
                        rep_ids=reps)
    ex = idx.export()
    o = oracle.build_oneshot(X, reps, s)
    r0 = int(np.nonzero(reps == 1000)[0][0])
    np.testing.assert_array_equal(ex["members"].reshape(-1, s)[r0], np.arange(1000, 1064))
    check_lists(X, reps, ex["members"], s, o.lists, "l2")
    Q = np.concatenate([X[1000:1001].repeat(5, 0), synth.iid_normal(200, 8, 2)]).astype(np.float32)
    ids, dist = search(idx, Q, 5)
    check_search(X, Q, o, ids, dist, 5, "l2")


@pytest.mark.parametrize("storage", ["bf16", "f16", "fp8"])
@pytest.mark.parametrize("k", [1, 10])
def test_oneshot_search_tensor_cores(storage, k):
    mod = synth.SubspaceModel(d=64, k=8, noise_var=0.01, seed=0)
    X = mod.sample(60000, 0)
    Q = mod.sample(3000, 1)
    n_r, s = 245, 700
    idx = build(X, n_r, s, storage={"bf16": rbc.BF16, "f16": rbc.F16, "fp8": rbc.FP8E4M3}[storage],
                seed=4)
    ids, dist = search(idx, Q, k)
    o = oracle.build_oneshot(X, oracle.sample_reps(len(X), n_r, 4), s)
    check_search(X, Q, o, ids, dist, k, "l2")


def test_oneshot_tensor_core_uncertified_rows_search_their_own_list():
    # queries exactly on 40 copies of a point: the low-precision scores of the
    # copies tie, certification fails, and the FP32 re-search must stay inside
    # the query's list (a search over every list would be a different answer)
    X = synth.iid_normal(20000, 32, 7)
    X[500:540] = X[100]
    Q = np.concatenate([X[100:101].repeat(64, 0), synth.iid_normal(400, 32, 8)]).astype(np.float32)
    n_r, s = 100, 300
    idx = build(X, n_r, s, storage=rbc.BF16, seed=11)
    ids, dist = search(idx, Q, 10)
    st = rbc.last_stats()
    assert st["uncertified"] >= 64
    o = oracle.build_oneshot(X, oracle.sample_reps(len(X), n_r, 11), s)
    check_search(X, Q, o, ids, dist, 10, "l2")


def test_oneshot_host_buffers_and_empty():
    X = synth.iid_normal(3000, 10, 1)
    Q = synth.iid_normal(130, 10, 2)
    idx = rbc.rbc_build(X, 40, mode=rbc.ONESHOT, s=90, seed=5)  # host X
    ids = np.empty((130, 4), dtype=np.int64)
    dist = np.empty((130, 4), dtype=np.float32)
    rbc.rbc_search(idx, Q, 4, out_ids=ids, out_dist=dist)  # host Q and outputs
    o = oracle.build_oneshot(X, oracle.sample_reps(3000, 40, 5), 90)
    check_search(X, Q, o, ids, dist, 4, "l2")
    e_ids, e_dist = rbc.rbc_search(idx, torch.zeros((0, 10), device="cuda"), 4)
    assert e_ids.shape == (0, 4) and e_dist.shape == (0, 4)


def test_oneshot_argument_errors():
    X = torch.from_numpy(synth.iid_normal(500, 4, 1)).cuda()
    with pytest.raises(rbc.RbcError):
        rbc.rbc_build(X, 10, mode=rbc.ONESHOT, s=0)
    with pytest.raises(rbc.RbcError):
        rbc.rbc_build(X, 10, mode=rbc.ONESHOT, s=501)
    idx = rbc.rbc_build(X, 10, mode=rbc.ONESHOT, s=20)
    with pytest.raises(rbc.RbcError):
        rbc.rbc_search(idx, X[:5], 21)  # k > s

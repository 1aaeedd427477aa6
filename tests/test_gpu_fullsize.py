"""Parity at full size.  Each workload is searched in one call over all of
its queries, as the benchmark launches it, and checked against the FP64
oracle on a seeded sample of queries (the oracle computes those one by one
against the whole database):

* 8-dim subspace of R^64, n = 2^20, 100,000 queries, n_r = 1024: exact and
  one-shot (s = n_r), L2 (BF16 and FP32) and L1;
* 1000 Gaussian clusters in R^128, n = 2^22, 65,536 queries, n_r = 2048,
  BF16, k = 10, top-32 FP32 re-rank;
* 12-dim sin/cos embedding in R^96, n = 2^23, n_r = 2896, FP16, k = 10
  (the resident index of the serving workload; 20,000 queries)."""
import numpy as np
import pytest

import oracle
import synth
from parity import TIE_REL, check_knn

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import paper_1103_2635_b300 as rbc  # noqa: E402

WL = "subspace8-n1m-d64"
SAMPLE = 2000


@pytest.fixture(scope="module")
def data():
    w = synth.WORKLOADS[WL]
    X, Q = synth.make_workload(w, seed=0)
    sel = np.sort(np.random.default_rng(11).choice(len(Q), SAMPLE, replace=False))
    return {
        "w": w,
        "X": X,
        "Q": Q,
        "Xd": torch.from_numpy(X).cuda(),
        "Qd": torch.from_numpy(Q).cuda(),
        "sel": sel,
        "oracle": {},
    }


def oracle_knn(data, metric, k=10):
    key = (metric, k)
    if key not in data["oracle"]:
        data["oracle"][key] = oracle.bf(data["Q"][data["sel"]], data["X"], k, metric)
    return data["oracle"][key]


def run(idx, data, k):
    ids, dist = rbc.rbc_search(idx, data["Qd"], k)
    torch.cuda.synchronize()
    sel = torch.from_numpy(data["sel"]).cuda()
    return ids[sel].cpu().numpy(), dist[sel].cpu().numpy()


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_fullsize_exact_l2(data, storage):
    st = {"bf16": rbc.BF16, "f32": rbc.F32}[storage]
    idx = rbc.rbc_build(data["Xd"], data["w"].n_r, metric=rbc.L2, seed=2, storage=st)
    o_ids, o_rho = oracle_knn(data, "l2")
    for k in (1, 10):
        ids, dist = run(idx, data, k)
        check_knn(data["Q"][data["sel"]], data["X"], ids, dist, o_ids[:, :k], o_rho[:, :k], "l2")


def test_fullsize_exact_l1(data):
    idx = rbc.rbc_build(data["Xd"], data["w"].n_r, metric=rbc.L1, seed=2)
    o_ids, o_rho = oracle_knn(data, "l1")
    for k in (1, 10):
        ids, dist = run(idx, data, k)
        check_knn(data["Q"][data["sel"]], data["X"], ids, dist, o_ids[:, :k], o_rho[:, :k], "l1")


@pytest.mark.parametrize("metric,storage", [("l2", "bf16"), ("l1", "f32")])
def test_fullsize_oneshot(data, metric, storage):
    w, X = data["w"], data["X"]
    s = w.n_r  # s = n_r
    st = {"bf16": rbc.BF16, "f32": rbc.F32}[storage]
    idx = rbc.rbc_build(data["Xd"], w.n_r, metric={"l2": rbc.L2, "l1": rbc.L1}[metric], seed=2,
                        mode=rbc.ONESHOT, s=s, storage=st)
    ex = idx.export()
    reps = oracle.sample_reps(len(X), w.n_r, 2)
    np.testing.assert_array_equal(ex["reps"], reps)
    lists = ex["members"].reshape(w.n_r, s)
    Qs = data["Q"][data["sel"]]
    # the oracle's nearest representative of every sampled query, and its list
    Dr = oracle.dist(Qs, X[reps], metric)
    near = np.argmin(Dr, axis=1)  # first minimum = smaller ordinal
    srt = np.sort(Dr, axis=1)
    amb = srt[:, 1] - srt[:, 0] <= TIE_REL * srt[:, 0]
    need = np.unique(near)
    o_l, o_lr = oracle.bf(X[reps[need]], X, s, metric)
    o_lists = {int(r): o_l[i] for i, r in enumerate(need)}
    # lists of the representatives the sample uses: equal up to FP64 near-ties
    for r in need[:: max(1, len(need) // 64)]:
        g, o = lists[r], o_lists[int(r)]
        if not np.array_equal(g, o):
            dg = oracle.dist(X[reps[r] : reps[r] + 1], X[g], metric)[0]
            np.testing.assert_allclose(dg, o_lr[np.searchsorted(need, r)], rtol=TIE_REL)
    for k in (1, 10):
        ids, dist = run(idx, data, k)
        ok = ~amb
        o_ids, o_rho = oracle.bf_lists(Qs[ok], X, [o_lists[int(r)] for r in near[ok]], k, metric)
        check_knn(Qs[ok], X, ids[ok], dist[ok], o_ids, o_rho, metric)
        assert ok.mean() > 0.99


@pytest.mark.parametrize("wl,storage,rerank_c,m,sample", [
    ("clusters1000-n4m-d128", "bf16", 32, None, 500),
    ("clusters1000-n4m-d128", "fp8", 32, None, 500),
    ("sincos12-n8m-d96", "f16", 0, 20000, 300),
])
def test_fullsize_exact_large(wl, storage, rerank_c, m, sample):
    w = synth.WORKLOADS[wl]
    X, Q = synth.make_workload(w, seed=0, m=m)
    sel = np.sort(np.random.default_rng(11).choice(len(Q), sample, replace=False))
    Xd = torch.from_numpy(X).cuda()
    st = {"bf16": rbc.BF16, "f16": rbc.F16, "fp8": rbc.FP8E4M3}[storage]
    idx = rbc.rbc_build(Xd, w.n_r, metric=rbc.L2, seed=2, storage=st, rerank_c=rerank_c)
    del Xd
    ids, dist = rbc.rbc_search(idx, torch.from_numpy(Q).cuda(), 10)
    torch.cuda.synchronize()
    ids, dist = ids.cpu().numpy()[sel], dist.cpu().numpy()[sel]
    idx.close()
    o_ids, o_rho = oracle.bf(Q[sel], X, 10, "l2")
    check_knn(Q[sel], X, ids, dist, o_ids, o_rho, "l2")

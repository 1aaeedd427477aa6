"""The grouped multi-index search (rbc_group_*): many independent exact
indexes of different sizes and dimensions searched together in one
persistent stage-two launch and one CUDA graph per batch shape.  Each index's
answer equals rbc_search on that index alone (ids outside near-ties of 1e-6
relative, distances within 1e-5 relative) and the FP64 oracle on sampled
rows."""
import numpy as np
import pytest

import oracle
import synth
from parity import DIST_REL, TIE_REL, check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402


def make_indexes(count, seed, storage=rbc.F16, nmax=30000, mmax=600, zero_m=True):
    """Indexes of the subspace model (each its own 8-dim subspace) with
    log-uniform sizes, dimensions from {32, 64, 96, 128}, ragged query counts."""
    rng = np.random.default_rng(seed)
    data = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(nmax))))
        d = int(rng.choice([32, 64, 96, 128]))
        m = int(np.exp(rng.uniform(np.log(1), np.log(mmax))))
        if zero_m and i == 1:
            m = 0
        mod = synth.SubspaceModel(d=d, k=8, noise_var=0.01, seed=1000 + i)
        X, Q = mod.sample(n, 2 * i), mod.sample(m, 2 * i + 1)
        idx = rbc.rbc_build(torch.from_numpy(X).cuda(), max(1, int(round(np.sqrt(n)))), seed=i,
                            storage=storage)
        data.append((X, Q, idx))
    torch.cuda.synchronize()
    return data


def alone(idx, Q, k):
    ids, dist = rbc.rbc_search(idx, torch.from_numpy(np.ascontiguousarray(Q)).cuda(), k)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def assert_same(ids, dist, ids_a, dist_a):
    np.testing.assert_allclose(dist, dist_a, rtol=DIST_REL, atol=0)
    diff = ids != ids_a
    if diff.any():
        da, db = dist[diff].astype(np.float64), dist_a[diff].astype(np.float64)
        assert np.all(np.abs(da - db) <= TIE_REL * np.maximum(db, 1e-30)), "ids differ outside a tie"


@pytest.mark.parametrize("storage,k", [(rbc.F16, 5), (rbc.BF16, 1), (rbc.F16, 10)])
def test_group_equals_each_index_alone_and_oracle(storage, k):
    data = make_indexes(12, seed=storage * 10 + k, storage=storage)
    with rbc.Group([ix for _, _, ix in data]) as g:
        Qs = [torch.from_numpy(Q).cuda() for _, Q, _ in data]
        ids, dist = g.search(Qs, k)
        torch.cuda.synchronize()
        st = g.stats()
    assert st["indexes"] == 12 and st["device_errors"] == 0
    assert st["queries"] == sum(len(Q) for _, Q, _ in data)
    for (X, Q, idx), gi, gd in zip(data, ids, dist):
        gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
        assert gi.shape == (len(Q), k)
        if len(Q) == 0:
            continue
        ia, da = alone(idx, Q, k)
        assert_same(gi, gd, ia, da)
        rows = np.unique(np.linspace(0, len(Q) - 1, min(len(Q), 20)).astype(int))
        o_ids, o_rho = oracle.bf(Q[rows], X, k)
        check_knn(Q[rows], X, gi[rows], gd[rows], o_ids, o_rho)
    for _, _, idx in data:
        idx.close()


def test_group_graph_replay_and_host_buffers():
    data = make_indexes(6, seed=3)
    with rbc.Group([ix for _, _, ix in data]) as g:
        Qs = [torch.from_numpy(Q).cuda() for _, Q, _ in data]
        g.search(Qs, 5)
        first = g.stats()["graph_replays"]
        # same shape, new values (host arrays): the graph is replayed
        rng = np.random.default_rng(0)
        Q2 = [Q + rng.normal(0, 0.05, Q.shape).astype(np.float32) for _, Q, _ in data]
        ids, dist = g.search(Q2, 5)
        assert g.stats()["graph_replays"] == first + 1
        for (X, _, idx), Q, gi, gd in zip(data, Q2, ids, dist):
            if len(Q):
                ia, da = alone(idx, Q, 5)
                assert_same(gi, gd, ia, da)
    for _, _, idx in data:
        idx.close()


def test_group_host_queries_per_index_equal_device():
    # host queries reach the library one pointer per index
    # (rbc_group_search_split, no packing on the host): pageable arrays and
    # pinned CPU tensors give the answers of device tensors (packed on the
    # device, rbc_group_search), index 1 with no queries at all
    data = make_indexes(7, seed=9)
    with rbc.Group([ix for _, _, ix in data]) as g:
        di, dd = g.search([torch.from_numpy(Q).cuda() for _, Q, _ in data], 5)
        torch.cuda.synchronize()
        hi, hd = g.search([Q for _, Q, _ in data], 5)
        pi, pd = g.search([torch.from_numpy(Q).pin_memory() for _, Q, _ in data], 5)
        for (_, Q, _), a, b, c, d, e, f in zip(data, di, dd, hi, hd, pi, pd):
            assert c.shape == (len(Q), 5) and e.shape == (len(Q), 5)
            np.testing.assert_array_equal(c, a.cpu().numpy())
            np.testing.assert_array_equal(d, b.cpu().numpy())
            np.testing.assert_array_equal(e, a.cpu().numpy())
            np.testing.assert_array_equal(f, b.cpu().numpy())
        # caller-owned pinned outputs are written in place
        M = sum(len(Q) for _, Q, _ in data)
        oi = torch.empty((M, 5), dtype=torch.int64).pin_memory()
        od = torch.empty((M, 5), dtype=torch.float32).pin_memory()
        qi, qd = g.search([torch.from_numpy(Q).pin_memory() for _, Q, _ in data], 5,
                          out_ids=oi, out_dist=od)
        np.testing.assert_array_equal(oi.numpy(), np.concatenate([a.cpu().numpy() for a in di]))
        np.testing.assert_array_equal(od.numpy(), np.concatenate([b.cpu().numpy() for b in dd]))
        for a, c in zip(di, qi):
            np.testing.assert_array_equal(c.numpy(), a.cpu().numpy())
        bad = [Q for _, Q, _ in data]
        bad[0] = np.zeros((3, data[0][1].shape[1] + 1), np.float32)
        with pytest.raises(ValueError):
            g.search(bad, 5)
        with pytest.raises(ValueError):  # outputs of the wrong size are refused
            g.search([Q for _, Q, _ in data], 5, out_ids=oi[:-1], out_dist=od[:-1])
    for _, _, idx in data:
        idx.close()


def test_group_autotune_keeps_results():
    data = make_indexes(8, seed=5, zero_m=False)
    with rbc.Group([ix for _, _, ix in data]) as g:
        Qs = [torch.from_numpy(Q).cuda() for _, Q, _ in data]
        ids0, dist0 = g.search(Qs, 5)
        W = g.tune(Qs, 5)
        assert W in (1024, 2048, 4096, 8192, 16384, 32768)
        ids1, dist1 = g.search(Qs, 5)
        assert g.stats()["work_item_points"] == W
        for a, b, c, d in zip(ids0, dist0, ids1, dist1):
            assert_same(c.cpu().numpy(), d.cpu().numpy(), a.cpu().numpy(), b.cpu().numpy())
    for _, _, idx in data:
        idx.close()


def test_group_rejects_unsupported_indexes():
    X = synth.iid_normal(2000, 16, 1)
    a = rbc.rbc_build(torch.from_numpy(X).cuda(), 40, storage=rbc.F16)
    b = rbc.rbc_build(torch.from_numpy(X).cuda(), 40, storage=rbc.BF16)
    c = rbc.rbc_build(torch.from_numpy(X).cuda(), 40, storage=rbc.F32)
    with pytest.raises(rbc.RbcError) as e:
        rbc.Group([a, b])
    assert e.value.code == -1
    with pytest.raises(rbc.RbcError) as e:
        rbc.Group([a, c])
    assert e.value.code == -5
    with rbc.Group([a]) as g:
        with pytest.raises(rbc.RbcError):
            g.search([np.zeros((3, 16), np.float32)], 0)
    for ix in (a, b, c):
        ix.close()

"""Parity of the CUDA brute-force primitive BF(Q, X) (Section 3) with the FP64
oracle, through the C ABI: FP32 CUDA-core path (l2, l1), ragged shapes,
degenerate inputs, host buffers."""
import numpy as np
import pytest

import oracle
import synth
from parity import check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

MET = {"l2": rbc.L2, "l1": rbc.L1}


def run_bf(Q, X, k, metric, storage=rbc.F32):
    Qd = torch.from_numpy(Q).cuda()
    Xd = torch.from_numpy(X).cuda()
    ids, dist = rbc.bf_search(Qd, Xd, k, metric=MET[metric], storage=storage)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("k", [1, 10])
def test_bf_iid_n16k_d16(metric, k):
    X, Q = synth.make_workload("iid-n16k-d16", seed=0)
    ids, dist = run_bf(Q, X, k, metric)
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("n,m,d,k", [(1000, 1, 3, 1), (4099, 129, 33, 5), (777, 300, 1, 7), (3000, 127, 100, 31), (2500, 257, 128, 3), (70000, 50, 64, 10), (65, 513, 256, 2)])
def test_bf_ragged(metric, n, m, d, k):
    X = synth.iid_normal(n, d, 1000 + n)
    Q = synth.iid_normal(m, d, 2000 + m)
    ids, dist = run_bf(Q, X, k, metric)
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


def test_bf_k_exceeds_n():
    X = synth.iid_normal(5, 8, 1)
    Q = synth.iid_normal(9, 8, 2)
    ids, dist = run_bf(Q, X, 8, "l2")
    o_ids, o_rho = oracle.bf(Q, X, 8, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)
    assert np.all(ids[:, 5:] == -1) and np.all(np.isinf(dist[:, 5:]))


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_bf_duplicates_and_ties(metric):
    base = synth.iid_normal(40, 6, 3)
    X = np.concatenate([base, base, base[:10], np.zeros((30, 6), np.float32)])
    Q = np.concatenate([base[:20], np.zeros((3, 6), np.float32), synth.iid_normal(20, 6, 4)])
    ids, dist = run_bf(Q, X, 6, metric)
    o_ids, o_rho = oracle.bf(Q, X, 6, metric)
    # exact duplicates give exactly equal distances: ids must follow (rho, id)
    np.testing.assert_array_equal(ids, o_ids)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


def test_bf_all_points_equal():
    X = np.ones((300, 4), np.float32)
    Q = synth.iid_normal(7, 4, 5)
    ids, dist = run_bf(Q, X, 4, "l2")
    np.testing.assert_array_equal(ids, np.tile(np.arange(4), (7, 1)))


def test_bf_empty_query_batch():
    X = synth.iid_normal(100, 4, 6)
    Q = np.zeros((0, 4), np.float32)
    ids, dist = run_bf(Q, X, 3, "l2")
    assert ids.shape == (0, 3)


def test_bf_host_buffers_match_device():
    X = synth.iid_normal(5000, 24, 7)
    Q = synth.iid_normal(300, 24, 8)
    h_ids, h_dist = rbc.bf_search(Q, X, 4)  # numpy in, numpy out
    d_ids, d_dist = run_bf(Q, X, 4, "l2")
    np.testing.assert_array_equal(h_ids, d_ids)
    np.testing.assert_array_equal(h_dist, d_dist)
    o_ids, o_rho = oracle.bf(Q, X, 4, "l2")
    check_knn(Q, X, h_ids, h_dist, o_ids, o_rho)


def test_bf_on_a_side_stream():
    X = synth.iid_normal(3000, 16, 9)
    Q = synth.iid_normal(200, 16, 10)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
        ids, dist = rbc.bf_search(Qd, Xd, 3)
    s.synchronize()
    o_ids, o_rho = oracle.bf(Q, X, 3, "l2")
    check_knn(Q, X, ids.cpu().numpy(), dist.cpu().numpy(), o_ids, o_rho)


# ---- tensor-core (tcgen05) path: bf16 / fp16 / FP8 E4M3 storage, FP32 re-rank, certified ----

LP = {"bf16": rbc.BF16, "f16": rbc.F16, "fp8": rbc.FP8E4M3}


@pytest.mark.parametrize("storage", ["bf16", "f16", "fp8"])
@pytest.mark.parametrize("k", [1, 10])
def test_bf_tc_iid_n16k_d16(storage, k):
    X, Q = synth.make_workload("iid-n16k-d16", seed=0)
    ids, dist = run_bf(Q, X, k, "l2", LP[storage])
    o_ids, o_rho = oracle.bf(Q, X, k, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)


@pytest.mark.parametrize("storage", ["bf16", "f16", "fp8"])
@pytest.mark.parametrize("n,m,d,k", [(1000, 1, 3, 1), (4099, 129, 33, 5), (3000, 127, 100, 31), (2500, 257, 128, 3), (70000, 300, 64, 10), (5000, 200, 200, 4), (600, 130, 256, 2)])
def test_bf_tc_ragged(storage, n, m, d, k):
    X = synth.iid_normal(n, d, 3000 + n)
    Q = synth.iid_normal(m, d, 4000 + m)
    ids, dist = run_bf(Q, X, k, "l2", LP[storage])
    o_ids, o_rho = oracle.bf(Q, X, k, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)


def test_bf_tc_subspace_workload():
    mod = synth.SubspaceModel(d=64, k=8, noise_var=0.01, seed=0)
    X = mod.sample(200000, 0)
    Q = mod.sample(1000, 1)
    for k in (1, 10):
        ids, dist = run_bf(Q, X, k, "l2", rbc.BF16)
        st = rbc.last_stats()
        o_ids, o_rho = oracle.bf(Q, X, k, "l2")
        check_knn(Q, X, ids, dist, o_ids, o_rho)
        assert st["uncertified"] <= 0.05 * len(Q), st


def test_bf_fp8_clusters_scales_and_certification():
    # clustered rows of very different magnitudes: each row gets its own
    # power-of-two scale; the scaled dequantisation error enters the bound,
    # uncertified queries are searched again in FP32, the answer stays exact
    mod = synth.ClusterModel(d=128, n_clusters=50, seed=3)
    X = mod.sample(30000, 0)
    X[:5000] *= 40.0
    X[5000:10000] *= 0.01
    Q = np.concatenate([mod.sample(300, 1), X[:50] * 1.001, X[5000:5050] * 0.999]).astype(np.float32)
    for k in (1, 10):
        ids, dist = run_bf(Q, X, k, "l2", rbc.FP8E4M3)
        o_ids, o_rho = oracle.bf(Q, X, k, "l2")
        check_knn(Q, X, ids, dist, o_ids, o_rho)


def test_bf_tc_duplicates_and_ties():
    base = synth.iid_normal(40, 6, 3)
    X = np.concatenate([base, base, base[:10], np.zeros((30, 6), np.float32)])
    Q = np.concatenate([base[:20], np.zeros((3, 6), np.float32), synth.iid_normal(20, 6, 4)])
    ids, dist = run_bf(Q, X, 6, "l2", rbc.BF16)
    o_ids, o_rho = oracle.bf(Q, X, 6, "l2")
    np.testing.assert_array_equal(ids, o_ids)


def test_bf_tc_k_exceeds_n_and_empty():
    X = synth.iid_normal(5, 8, 1)
    Q = synth.iid_normal(9, 8, 2)
    ids, dist = run_bf(Q, X, 8, "l2", rbc.BF16)
    o_ids, o_rho = oracle.bf(Q, X, 8, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho)
    ids, dist = run_bf(np.zeros((0, 8), np.float32), X, 2, "l2", rbc.BF16)
    assert ids.shape == (0, 2)

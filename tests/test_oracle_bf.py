"""Pins for the oracle's brute-force primitive BF(Q, X) (Section 3).

Each check is independent of the oracle's own code: scipy's k-d tree (a
library k-NN), a Python enumeration built on ``math.dist`` / ``sum(abs)``,
and the integer-lattice closed form (the l1 lattice of Section 6).
"""
import itertools
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import synth


@pytest.mark.parametrize("metric,p", [("l2", 2), ("l1", 1)])
@pytest.mark.parametrize("n,m,d,k", [(500, 40, 3, 1), (1000, 30, 8, 10), (257, 17, 16, 5), (64, 9, 1, 7)])
def test_bf_matches_kdtree(metric, p, n, m, d, k):
    X = synth.iid_normal(n, d, seed=11 + d)
    Q = synth.iid_normal(m, d, seed=12 + d)
    ids, rho = oracle.bf(Q, X, k, metric)
    tree = cKDTree(X.astype(np.float64))
    kd_rho, kd_ids = tree.query(Q.astype(np.float64), k=k, p=p)
    kd_rho = kd_rho.reshape(m, k)
    kd_ids = kd_ids.reshape(m, k)
    np.testing.assert_array_equal(ids, kd_ids)
    np.testing.assert_allclose(rho, kd_rho, rtol=1e-12, atol=1e-12)


def _enumerate(Q, X, k, metric):
    out_ids, out_rho = [], []
    for q in Q.astype(np.float64):
        if metric == "l2":
            rs = [math.dist(q, x) for x in X.astype(np.float64)]
        else:
            rs = [sum(abs(a - b) for a, b in zip(q, x)) for x in X.astype(np.float64)]
        order = sorted(range(len(X)), key=lambda i: (rs[i], i))[:k]
        out_ids.append(order)
        out_rho.append([rs[i] for i in order])
    return np.array(out_ids), np.array(out_rho)


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_bf_enumeration_tiny(metric):
    X = synth.iid_normal(23, 4, seed=5)
    Q = synth.iid_normal(6, 4, seed=6)
    for k in (1, 3, 23):
        ids, rho = oracle.bf(Q, X, k, metric)
        e_ids, e_rho = _enumerate(Q, X, k, metric)
        np.testing.assert_array_equal(ids, e_ids)
        np.testing.assert_allclose(rho, e_rho, rtol=1e-14)


def test_bf_ties_break_by_id():
    # three copies of one point and two copies of another: equal rho -> smaller id
    p = np.array([1.0, 2.0, 3.0], np.float32)
    r = np.array([1.0, 2.0, 4.0], np.float32)
    X = np.stack([r, p, r, p, p, np.array([9, 9, 9], np.float32)])
    Q = p[None, :]
    for metric in ("l2", "l1"):
        ids, rho = oracle.bf(Q, X, 6, metric)
        assert ids[0].tolist() == [1, 3, 4, 0, 2, 5]
        assert rho[0, :3].tolist() == [0.0, 0.0, 0.0]
        assert rho[0, 3] == rho[0, 4] == 1.0


def test_bf_query_equidistant_pair():
    # q at the midpoint of x0=(2,0) and x1=(0,0): equal distance 1, id order
    X = np.array([[2.0, 0.0], [0.0, 0.0], [5.0, 5.0]], np.float32)
    Q = np.array([[1.0, 0.0]], np.float32)
    ids, rho = oracle.bf(Q, X, 2, "l2")
    assert ids.tolist() == [[0, 1]] and rho.tolist() == [[1.0, 1.0]]


def test_bf_k_beyond_n_pads():
    X = synth.iid_normal(3, 2, seed=1)
    ids, rho = oracle.bf(X[:1], X, 5, "l2")
    assert ids[0, 3:].tolist() == [-1, -1] and np.isinf(rho[0, 3:]).all()


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_grid_closed_form(metric, d):
    """On the lattice {0..G-1}^d the nearest point to an interior off-lattice
    query is its coordinate-wise rounding (unique when no fractional part is
    1/2), under both l1 and l2.  The second nearest differs from it in the one
    coordinate whose fractional part is closest to 1/2, moved to the other
    side; its distance follows in closed form."""
    G = 6 if d <= 3 else 5
    X = synth.grid_points(G, d)
    g = np.random.default_rng(100 + d)
    Q = g.uniform(1.0, G - 2.0, size=(64, d)).astype(np.float32)
    frac = Q - np.floor(Q)
    ok = np.all(np.abs(frac - 0.5) > 1e-3, axis=1)
    # the two coordinates closest to 1/2 must differ for the 2nd-NN to be unique
    dist_half = np.sort(np.abs(frac - 0.5), axis=1)
    if d > 1:
        ok &= (dist_half[:, 1] - dist_half[:, 0]) > 1e-3
    Q = Q[ok]
    ids, rho = oracle.bf(Q, X, 2, metric)
    R1 = np.rint(Q).astype(np.int64)
    strides = G ** np.arange(d - 1, -1, -1)
    np.testing.assert_array_equal(ids[:, 0], R1 @ strides)
    q64 = Q.astype(np.float64)
    if metric == "l2":
        exp1 = np.sqrt(((q64 - R1) ** 2).sum(1))
    else:
        exp1 = np.abs(q64 - R1).sum(1)
    np.testing.assert_allclose(rho[:, 0], exp1, rtol=1e-12)
    # second nearest
    j = np.argmin(np.abs(Q - np.floor(Q) - 0.5), axis=1)
    R2 = R1.copy()
    rows = np.arange(len(Q))
    R2[rows, j] += np.where(Q[rows, j] > R1[rows, j], 1, -1)
    np.testing.assert_array_equal(ids[:, 1], R2 @ strides)


def test_dist_matrix_matches_bf():
    X = synth.iid_normal(50, 5, seed=3)
    Q = synth.iid_normal(7, 5, seed=4)
    for metric in ("l2", "l1"):
        D = oracle.dist(Q, X, metric)
        ids, rho = oracle.bf(Q, X, 50, metric)
        np.testing.assert_array_equal(np.take_along_axis(D, ids, 1), rho)
        tree_p = 2 if metric == "l2" else 1
        ref = np.array([[np.linalg.norm(q.astype(np.float64) - x.astype(np.float64), ord=tree_p) for x in X] for q in Q])
        np.testing.assert_allclose(D, ref, rtol=1e-13)


def test_bf_lists_restricts_search():
    X = synth.iid_normal(200, 6, seed=8)
    Q = synth.iid_normal(5, 6, seed=9)
    lists = [np.arange(0, 200, s + 2) for s in range(5)]
    ids, rho = oracle.bf_lists(Q, X, lists, 4, "l2")
    tree_ids = []
    for i, l in enumerate(lists):
        sub = X[l].astype(np.float64)
        _, loc = cKDTree(sub).query(Q[i].astype(np.float64), k=4)
        tree_ids.append(l[loc])
    np.testing.assert_array_equal(ids, np.array(tree_ids))


def test_thread_count_does_not_change_result():
    X = synth.iid_normal(3000, 8, seed=21)
    Q = synth.iid_normal(64, 8, seed=22)
    a = oracle.bf(Q, X, 7, "l2", threads=1)
    b = oracle.bf(Q, X, 7, "l2", threads=0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])

"""Pins for the oracle's Random Ball Cover (Sections 4-6).

* Exact search returns exactly the brute-force neighbours, for every seed,
  n_r, k and metric: Section 5 states the exact algorithm is always correct
  and only its running time is random.
* Lemma 1 (Section 6 / Appendix A): the representative owning q's nearest
  neighbour lies within 3 gamma of q.
* Claim 2 (Section 6.1): the nearest neighbour lies within 4 gamma of its own
  representative and within 7 gamma of q.
* Exact lists partition X and every point lies within psi of its owner
  (Section 4), and the owner is a nearest representative (checked against
  scipy's k-d tree).
* Claim 1 (Section 6.1): E|B(q, gamma)| = n / n_r under independent selection;
  with exactly n_r distinct representatives drawn uniformly, the count of
  points strictly closer than the nearest representative has mean
  (n - n_r) / (n_r + 1) (the first success among n_r marked positions of a
  random permutation of n).
* One-shot lists are exactly the s nearest points of each representative
  (Section 5.1), checked against scipy's k-d tree.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import synth


def _data(n, m, d, seed):
    return synth.iid_normal(n, d, seed), synth.iid_normal(m, d, seed + 1)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("n,d,n_r,k,seed", [(2000, 4, 45, 1, 0), (2000, 4, 45, 10, 1), (3000, 8, 55, 3, 2), (500, 2, 500, 5, 3), (400, 3, 3, 7, 4), (300, 5, 1, 2, 5)])
def test_exact_search_equals_bf(metric, n, d, n_r, k, seed):
    X, Q = _data(n, 60, d, seed)
    reps = oracle.sample_reps(n, n_r, seed + 2)
    idx = oracle.build_exact(X, reps, metric)
    ids, rho, st = oracle.search_exact(idx, Q, k)
    bids, brho = oracle.bf(Q, X, k, metric)
    np.testing.assert_array_equal(ids, bids)
    np.testing.assert_array_equal(rho, brho)
    assert np.all(st.examined >= k) or n < k


def test_exact_search_with_duplicates_equals_bf():
    # many exact duplicates, including duplicated representatives
    base = synth.iid_normal(50, 3, 7)
    X = np.concatenate([base, base, base[:20], base[:5]])
    Q = np.concatenate([base[:10], synth.iid_normal(20, 3, 8)])
    for n_r in (1, 7, 40, len(X)):
        reps = oracle.sample_reps(len(X), n_r, 11)
        idx = oracle.build_exact(X, reps, "l2")
        for k in (1, 4):
            ids, rho, _ = oracle.search_exact(idx, Q, k)
            bids, brho = oracle.bf(Q, X, k, "l2")
            np.testing.assert_array_equal(ids, bids)


@pytest.mark.parametrize("metric,p", [("l2", 2), ("l1", 1)])
def test_build_partition_radius_and_owner(metric, p):
    X, _ = _data(4000, 1, 6, 20)
    reps = oracle.sample_reps(len(X), 63, 22)
    idx = oracle.build_exact(X, reps, metric)
    allids = np.sort(np.concatenate(idx.lists))
    np.testing.assert_array_equal(allids, np.arange(len(X)))
    for r, l in enumerate(idx.lists):
        assert np.all(idx.owner[l] == r)
        assert np.all(np.diff(l) > 0)
        if len(l):
            assert idx.psi[r] == idx.owner_rho[l].max()
        else:
            assert idx.psi[r] == 0.0
        # a representative owns itself unless a duplicate with a smaller id exists
        assert r == idx.owner[reps[r]] or idx.owner_rho[reps[r]] == 0.0
    # owner is a nearest representative: compare its distance with a k-d tree
    tree = cKDTree(X[reps].astype(np.float64))
    kd_rho, _ = tree.query(X.astype(np.float64), k=1, p=p)
    np.testing.assert_allclose(idx.owner_rho, kd_rho, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_lemma1_and_claim2(metric):
    X, Q = _data(5000, 200, 5, 30)
    reps = oracle.sample_reps(len(X), 70, 32)
    idx = oracle.build_exact(X, reps, metric)
    D = oracle.dist(Q, X[reps], metric)
    gamma = D.min(axis=1)
    nn, nn_rho = oracle.bf(Q, X, 1, metric)
    owner = idx.owner[nn[:, 0]]
    rho_q_owner = D[np.arange(len(Q)), owner]
    assert np.all(rho_q_owner <= 3.0 * gamma * (1 + 1e-12))  # Lemma 1
    assert np.all(idx.owner_rho[nn[:, 0]] <= 4.0 * gamma * (1 + 1e-12))  # within 4 gamma of its rep
    assert np.all(nn_rho[:, 0] <= 7.0 * gamma * (1 + 1e-12))  # Claim 2: inside B(q, 7 gamma)
    assert np.all(nn_rho[:, 0] <= gamma)  # gamma bounds the NN distance (r_q is in X)


def test_claim1_expected_ball_size():
    n, n_r, d = 3000, 30, 3
    X = synth.iid_normal(n, d, 40)
    Q = synth.iid_normal(40, d, 41)
    Dall = oracle.dist(Q, X, "l2")
    counts = []
    for s in range(60):
        reps = oracle.sample_reps(n, n_r, 500 + s)
        gamma = Dall[:, reps].min(axis=1)
        counts.extend((Dall < gamma[:, None]).sum(axis=1).tolist())
    counts = np.array(counts, dtype=np.float64)
    expect = (n - n_r) / (n_r + 1)
    # geometric-like law: sd ~ mean; queries share reps per seed, so use the
    # seed means (60 independent draws) for the standard error
    seed_means = counts.reshape(60, -1).mean(axis=1)
    se = seed_means.std(ddof=1) / np.sqrt(len(seed_means))
    assert abs(seed_means.mean() - expect) < 4 * se, (seed_means.mean(), expect, se)
    # the paper's n / n_r is the independent-selection value; both agree to O(1/n_r)
    assert abs(expect - n / n_r) / (n / n_r) < 0.05


@pytest.mark.parametrize("metric,p", [("l2", 2), ("l1", 1)])
def test_oneshot_lists_are_s_nearest(metric, p):
    X, Q = _data(3000, 100, 4, 50)
    reps = oracle.sample_reps(len(X), 40, 52)
    s = 40
    idx = oracle.build_oneshot(X, reps, s, metric)
    tree = cKDTree(X.astype(np.float64))
    kd_rho, kd_ids = tree.query(X[reps].astype(np.float64), k=s, p=p)
    np.testing.assert_array_equal(idx.lists, kd_ids)
    np.testing.assert_allclose(idx.psi, kd_rho[:, -1], rtol=1e-12)
    assert np.all(idx.lists[:, 0] == reps)  # rho(r, r) = 0 and no duplicates here
    ids, rho, near = oracle.search_oneshot(idx, Q, 3)
    # the searched list is that of the nearest representative
    D = oracle.dist(Q, X[reps], metric)
    np.testing.assert_array_equal(near, D.argmin(axis=1))
    for i in range(len(Q)):
        l = idx.lists[near[i]]
        sub = oracle.dist(Q[i : i + 1], X[l], metric)[0]
        order = np.lexsort((l, sub))[:3]
        np.testing.assert_array_equal(ids[i], l[order])


def test_oneshot_finds_nn_when_query_is_close_to_its_rep():
    """Appendix B: if rho(q, r) <= psi_r / 2 then q's nearest neighbour is in L_r."""
    X, Q = _data(4000, 300, 3, 60)
    reps = oracle.sample_reps(len(X), 60, 62)
    idx = oracle.build_oneshot(X, reps, 60, "l2")
    ids, rho, near = oracle.search_oneshot(idx, Q, 1)
    D = oracle.dist(Q, X[reps], "l2")
    close = D[np.arange(len(Q)), near] <= idx.psi[near] / 2
    bids, brho = oracle.bf(Q, X, 1, "l2")
    assert close.sum() > 20
    np.testing.assert_array_equal(ids[close, 0], bids[close, 0])


def test_rank_of_exact_answer_is_zero():
    X, Q = _data(500, 10, 3, 70)
    ids, _ = oracle.bf(Q, X, 2, "l2")
    assert np.all(oracle.rank_of(Q, X, ids[:, 0]) == 0)
    assert np.all(oracle.rank_of(Q, X, ids[:, 1]) == 1)


def test_planted_mistake_is_caught():
    """A pruning rule with a dropped term (gamma_k + psi_r replaced by psi_r)
    must make exact search disagree with BF somewhere; this checks that the
    equality test above has teeth."""
    X, Q = _data(3000, 200, 4, 80)
    reps = oracle.sample_reps(len(X), 50, 82)
    idx = oracle.build_exact(X, reps, "l2")
    D = oracle.dist(Q, X[reps], "l2")
    bids, _ = oracle.bf(Q, X, 1, "l2")
    keep_bad = D <= idx.psi[None, :]
    lists = [np.concatenate([idx.lists[r] for r in np.nonzero(kb)[0]] or [np.zeros(0, np.int64)]) for kb in keep_bad]
    lists = [l if len(l) else np.array([0]) for l in lists]
    ids_bad, _ = oracle.bf_lists(Q, X, lists, 1, "l2")
    assert np.any(ids_bad[:, 0] != bids[:, 0])

"""Parity rule between the CUDA path and the FP64 oracle.

Ids must match the oracle's exactly, except where the oracle itself has a
near-tie: a returned id may differ from the oracle's at rank j only if its
true (FP64) distance lies within ``tie_rel`` (relative) of the oracle's rank-j
distance, and the returned set must still be a valid k-NN set (distinct ids,
each no farther than the oracle's k-th distance times (1 + tie_rel)).
Distances must agree with the oracle's within ``dist_rel`` relative.
"""
import numpy as np

import oracle

TIE_REL = 1e-6
DIST_REL = 1e-5


def check_knn(Q, X, ids, dist, o_ids, o_rho, metric="l2", tie_rel=TIE_REL, dist_rel=DIST_REL):
    ids = np.asarray(ids)
    dist = np.asarray(dist, dtype=np.float64)
    m, k = o_ids.shape
    assert ids.shape == (m, k) and dist.shape == (m, k)
    valid = o_ids >= 0
    np.testing.assert_array_equal(ids[~valid], -1)
    assert np.all(np.isinf(dist[~valid]))
    ok_d = np.abs(dist[valid] - o_rho[valid]) <= dist_rel * np.maximum(o_rho[valid], 1e-30) + 1e-30
    if not ok_d.all():
        bad = np.argwhere(~ok_d)[:5]
        raise AssertionError(f"distance mismatch at {bad}: {dist[valid][~ok_d][:5]} vs {o_rho[valid][~ok_d][:5]}")
    exceptions = 0
    for i in np.nonzero(np.any(ids != o_ids, axis=1))[0]:
        row = ids[i][valid[i]]
        assert len(set(row.tolist())) == len(row), f"duplicate ids in row {i}: {row}"
        true = oracle.dist(Q[i : i + 1], X[row], metric)[0]
        kth = o_rho[i][valid[i]][-1]
        assert np.all(true <= kth * (1 + tie_rel) + 1e-30), f"row {i}: returned point beyond the k-th distance"
        for j in np.nonzero(ids[i] != o_ids[i])[0]:
            assert abs(true[j] - o_rho[i, j]) <= tie_rel * max(o_rho[i, j], 1e-30) + 1e-30, (
                f"row {i} rank {j}: id {ids[i, j]} (rho {true[j]}) vs oracle {o_ids[i, j]} (rho {o_rho[i, j]})"
            )
        exceptions += 1
    return exceptions

"""Rows that the FP32 certificate cannot decide, checked against the FP64 oracle.

Each test query gets a shell of points at distances R (1 + j g), j = 0, 1, ...,
with relative gaps g between the 1e-6 tie threshold of the parity rule and
the FP32 rounding bound of the select step: the FP64 order of the shell is
fixed, but the FP32 candidate set cannot certify it, so the query has to be
finished exactly (the FP64 band pass -- a few rows split over several CTAs,
many rows one CTA each -- or the FP64 band finish of the windowed select).  The tests assert that such rows occurred (the
`uncertified` / `boundary_ties` counters) and that every answer matches the
oracle element by element (Section 3: BF returns the k nearest; Section 5.2:
the exact search is always correct)."""
import numpy as np
import pytest

import oracle
from parity import check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1103_2635_b300 as rbc  # noqa: E402

MET = {"l2": rbc.L2, "l1": rbc.L1}


def shell_inputs(d, metric, n_bg=20000, m=48, shelled=16, J=48, gap=1.6e-6, dups=0, seed=7):
    """Queries Q [m, d]; database = background points far away plus, for each
    of the first `shelled` queries, J points at distances R (1 + j gap) in
    random directions (and `dups` exact copies of that query's shell point
    at j = 9, so that equal distances meet the 10th place)."""
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((m, d)).astype(np.float32)
    bg = (rng.standard_normal((n_bg, d)) * 3.0).astype(np.float32)
    pts = []
    for i in range(shelled):
        R = 0.5 + 0.25 * rng.random()
        v = rng.standard_normal((J, d))
        norm = np.abs(v).sum(1) if metric == "l1" else np.sqrt((v * v).sum(1))
        v /= norm[:, None]
        r = R * (1.0 + gap * np.arange(J))
        shell = (Q[i].astype(np.float64) + r[:, None] * v).astype(np.float32)
        pts.append(shell)
        if dups:
            pts.append(np.repeat(shell[9:10], dups, axis=0))
    X = np.concatenate([bg] + pts)
    X = X[rng.permutation(len(X))]
    return np.ascontiguousarray(X), Q


def _cpu(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("d,k", [(64, 31), (64, 30), (256, 24)])
def test_bf_f32_uncertified_rows_match_oracle(metric, d, k):
    X, Q = shell_inputs(d, metric)
    Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
    ids, dist = rbc.bf_search(Qd, Xd, k, metric=MET[metric], storage=rbc.F32)
    ids, dist = _cpu(ids), _cpu(dist)
    st = rbc.last_stats()
    assert st["uncertified"] > 0, st
    o_ids, o_rho = oracle.bf(Q, X, k, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_bf_f32_many_uncertified_rows_match_oracle(metric):
    # more uncertified rows than the band pass splits across CTAs (64): the
    # rows are then scanned whole, one CTA each
    X, Q = shell_inputs(48, metric, n_bg=20000, m=160, shelled=120, seed=9)
    Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
    ids, dist = rbc.bf_search(Qd, Xd, 31, metric=MET[metric], storage=rbc.F32)
    ids, dist = _cpu(ids), _cpu(dist)
    st = rbc.last_stats()
    assert st["uncertified"] > 64, st
    o_ids, o_rho = oracle.bf(Q, X, 31, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("metric", ["l2", "l1"])
def test_bf_noalloc_uncertified_rows_match_oracle(metric):
    X, Q = shell_inputs(64, metric)
    Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
    for _ in range(2):  # the static scratch keeps the previous call's contents
        ids, dist = rbc.bf_search_noalloc(Qd, Xd, 31, metric=MET[metric])
        ids, dist = _cpu(ids), _cpu(dist)
        st = rbc.last_stats()
        assert st["uncertified"] > 0 and st["queries"] == len(Q), st
        o_ids, o_rho = oracle.bf(Q, X, 31, metric)
        check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("metric", ["l2", "l1"])
@pytest.mark.parametrize("plan", [rbc.PLAN_WINDOW, rbc.PLAN_TILE_UNION])
def test_exact_search_f32_uncertified_rows_match_oracle(metric, plan):
    # tile-union plan: the FP32 certificate fails and the FP64 band pass
    # finishes the rows; windowed plan: every survivor in the tie band of the
    # k-th place is decided in FP64 by the select step
    X, Q = shell_inputs(64, metric)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    idx = rbc.rbc_build(Xd, 128, metric=MET[metric], seed=3, storage=rbc.F32, plan=plan)
    ids, dist = rbc.rbc_search(idx, Qd, 31)
    ids, dist = _cpu(ids), _cpu(dist)
    st = rbc.last_stats()
    idx.close()
    if plan == rbc.PLAN_TILE_UNION:
        assert st["uncertified"] > 0, st
    else:
        assert st["boundary_ties"] > 0, st
    o_ids, o_rho = oracle.bf(Q, X, 31, metric)
    check_knn(Q, X, ids, dist, o_ids, o_rho, metric)


@pytest.mark.parametrize("plan", [rbc.PLAN_WINDOW, rbc.PLAN_TILE_UNION])
@pytest.mark.parametrize("k", [10, 31])
def test_exact_search_bf16_shell_matches_oracle(plan, k):
    # low-precision storage: the shell's tie band reaches past the k-th place
    # in the re-ranked candidates (windowed plan: the FP64 band finish of the
    # select; tile-union plan: re-search, then the FP64 band pass)
    X, Q = shell_inputs(64, "l2", gap=1.2e-6, dups=40)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    idx = rbc.rbc_build(Xd, 128, seed=3, storage=rbc.BF16, plan=plan)
    ids, dist = rbc.rbc_search(idx, Qd, k)
    ids, dist = _cpu(ids), _cpu(dist)
    st = rbc.last_stats()
    idx.close()
    assert st["boundary_ties"] + st["uncertified"] > 0, st
    o_ids, o_rho = oracle.bf(Q, X, k, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho, "l2")


def test_bf_f32_equidistant_duplicates_past_the_list_width():
    # 40 exact copies at the 10th place: FP64 ties, ordered by id
    X, Q = shell_inputs(32, "l2", gap=2e-6, dups=40)
    Qd, Xd = torch.from_numpy(Q).cuda(), torch.from_numpy(X).cuda()
    ids, dist = rbc.bf_search(Qd, Xd, 10, metric=rbc.L2, storage=rbc.F32)
    ids, dist = _cpu(ids), _cpu(dist)
    o_ids, o_rho = oracle.bf(Q, X, 10, "l2")
    check_knn(Q, X, ids, dist, o_ids, o_rho, "l2")
    # the first 9 shell points are FP64-distinct (gaps above the tie rule)
    np.testing.assert_array_equal(ids[:16, :9], o_ids[:16, :9])

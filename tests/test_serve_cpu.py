"""Host-side checks of the serving engine's admission rule (rbc_plan_batch):
requests leave the queue in arrival order, a batch holds at most max_batch
queries, and it is shrunk until its workspace bound fits the memory left."""
import numpy as np
import pytest

import paper_1103_2635_b300 as rbc


def test_takes_whole_queue_when_it_fits():
    assert rbc.plan_batch([5, 7, 1], [1, 10, 5], max_batch=100, mem_left=1 << 40) == 3


def test_stops_at_max_batch_in_arrival_order():
    # 100 + 200 + 300 = 600 <= 1000, adding 4000 would exceed: the later small
    # request is not pulled past the large one (first come, first served)
    assert rbc.plan_batch([100, 200, 300, 4000, 1], [1] * 5, max_batch=1000, mem_left=1 << 40) == 3
    assert rbc.plan_batch([1000, 1], [1, 1], max_batch=1000, mem_left=1 << 40) == 1


def test_shrinks_to_the_memory_left():
    m, k = [100, 200, 300], [1, 10, 5]
    fixed, per_q, per_qk = 1000, 100, 10
    # bound(c) = fixed + queries * (per_q + max k * per_qk)
    b = [fixed + 100 * (100 + 10), fixed + 300 * (100 + 100), fixed + 600 * (100 + 100)]
    for left, want in [(b[2], 3), (b[2] - 1, 2), (b[1], 2), (b[1] - 1, 1), (b[0], 1), (b[0] - 1, 0)]:
        assert rbc.plan_batch(m, k, 10_000, left, fixed, per_q, per_qk) == want


def test_largest_k_of_the_batch_sets_its_bound():
    # the second request's k = 30 makes a two-request batch cost 2 x 31 per query
    m, k = [10, 10], [1, 30]
    assert rbc.plan_batch(m, k, 100, 20 * (1 + 30), 0, 1, 1) == 2
    assert rbc.plan_batch(m, k, 100, 20 * (1 + 30) - 1, 0, 1, 1) == 1


def test_empty_queue_and_bad_arguments():
    assert rbc.plan_batch([], [], 10, 1 << 30) == 0
    with pytest.raises(rbc.RbcError):
        rbc.plan_batch([1], [1], 0, 1 << 30)


@pytest.mark.parametrize("seed", range(5))
def test_random_queues_against_the_rule(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    m = np.exp(rng.uniform(0, np.log(4096), n)).astype(np.int64)
    k = rng.integers(1, 31, n).astype(np.int32)
    max_batch = int(rng.integers(4096, 20000))
    fixed, per_q, per_qk = int(rng.integers(0, 1 << 20)), int(rng.integers(1, 5000)), int(rng.integers(0, 100))
    left = int(rng.integers(0, 1 << 28))
    c = rbc.plan_batch(m, k, max_batch, left, fixed, per_q, per_qk)

    def bound(j):
        return fixed + int(m[:j].sum()) * (per_q + int(k[:j].max()) * per_qk)

    assert 0 <= c <= n
    if c:
        assert m[:c].sum() <= max_batch and bound(c) <= left
    # c is the largest prefix within max_batch whose bound fits
    j = c + 1
    if j <= n and m[:j].sum() <= max_batch:
        assert bound(j) > left

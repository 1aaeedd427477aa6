"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function that include/rbc.h declares, validates arguments, and its
representative sampler agrees with the oracle's independent one."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1103_2635_b300 as rbc

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rbc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("rbc_build", "rbc_search", "bf_search", "rbc_free", "rbc_last_error", "rbc_sample_reps"):
        assert f in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(rbc.library_path())
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


@pytest.mark.parametrize("n,n_r,seed", [(16384, 128, 2), (1 << 20, 1024, 2), (10, 10, 0), (7, 1, 3), (1 << 22, 2048, 2), (100003, 317, 12345)])
def test_sampler_matches_oracle(n, n_r, seed):
    np.testing.assert_array_equal(rbc.rbc_sample_reps(n, n_r, seed), oracle.sample_reps(n, n_r, seed))


def test_sampler_rejects_bad_args():
    for n, n_r in [(0, 1), (5, 0), (5, 6)]:
        with pytest.raises(rbc.RbcError) as e:
            rbc.rbc_sample_reps(n, n_r, 0)
        assert e.value.code == -1


def test_argument_validation_without_device_work():
    Q = np.zeros((2, 3), np.float32)
    X = np.zeros((4, 3), np.float32)
    for kw in [dict(k=0), dict(k=40)]:
        with pytest.raises(rbc.RbcError):
            rbc.bf_search(Q, X, **kw)
    with pytest.raises(rbc.RbcError) as e:
        rbc.bf_search(Q, X, 1, metric=7)
    assert e.value.code == -1
    with pytest.raises(rbc.RbcError) as e:
        rbc.bf_search(Q, X, 1, storage=9)
    assert e.value.code == -1
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_build(X, n_r=5)
    assert e.value.code == -1
    with pytest.raises(rbc.RbcError) as e:
        rbc.rbc_build(X, n_r=2, rep_ids=[3, 1])
    assert e.value.code == -1
    wide = np.zeros((4, 300), np.float32)
    with pytest.raises(rbc.RbcError) as e:
        rbc.bf_search(wide[:1], wide, 1)
    assert e.value.code == -5


def test_group_entries_reject_null_arguments_without_device_work():
    lib = rbc.load()
    # a NULL group, or a NULL array of per-index query pointers: RBC_ERR_ARG
    # before any CUDA call
    assert lib.rbc_group_search(None, None, None, 5, None, None, None) == -1
    assert lib.rbc_group_search_split(None, None, None, 5, None, None, None) == -1


def test_caller_output_buffers_are_checked_before_use():
    # Group.search writes into caller-owned outputs in place: a buffer of the
    # wrong shape, or one that would need a converted copy, is refused
    p, dev = rbc._check_out(np.empty((3, 5), np.int64), np.int64, 3, 5)
    assert p and not dev
    with pytest.raises(ValueError):
        rbc._check_out(np.empty((2, 5), np.int64), np.int64, 3, 5)
    with pytest.raises(TypeError):
        rbc._check_out(np.empty((3, 5), np.int32), np.int64, 3, 5)
    with pytest.raises(TypeError):
        rbc._check_out(np.empty((5, 3), np.int64).T, np.int64, 3, 5)

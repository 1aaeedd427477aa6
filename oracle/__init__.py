"""CPU oracle for the Random Ball Cover (Cayton, "Accelerating Nearest Neighbor
Search on Manycore Systems").

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs do.  It shares no code with the CUDA library;
inputs come from ``synth`` (random draws only).

Contents, each following the paper's definitions in the paper's order:

* :func:`bf`          -- the brute-force primitive BF(Q, X) (Section 3), FP64,
                         k smallest (rho, id) pairs; plain C in ``bf_ref.c``.
* :func:`dist`        -- every rho(q, x) (needed by the exact search, which
                         keeps all representative distances; Section 5.2).
* :func:`bf_lists`    -- BF(Q, X[L]) for a per-query id list (Section 3).
* :func:`sample_reps` -- the representative set R (Section 4), read as exactly
                         n_r distinct ids drawn without replacement by a
                         partial Fisher-Yates shuffle driven by SplitMix64
                         (Steele, Lea & Flood 2014), returned sorted.
* :func:`build_exact`, :func:`search_exact`     -- Section 4 / Section 5.2.
* :func:`build_oneshot`, :func:`search_oneshot` -- Section 4 / Section 5.1.

Pins (see ``tests/test_oracle_*.py``): BF against scipy's k-d tree and a
Python enumeration; the integer-lattice closed form (the lattice example of
Section 6); SplitMix64's published output stream; exact search equal to BF
(Section 5: the exact algorithm is always correct); Lemma 1, the 4-gamma and
7-gamma claims of Section 6.1; Claim 1's expected |B(q, gamma)|; one-shot
lists equal to the s nearest points of each representative.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_ref.c")
_LIB_PATH = os.path.join(_HERE, "libbf_ref.so")
_lib = None

L2, L1 = 0, 1
_METRICS = {"l2": L2, "l1": L1, L2: L2, L1: L1}


def build_lib(force: bool = False) -> str:
    """Compile ``bf_ref.c`` into ``libbf_ref.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        p = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_bf.argtypes = [p, i64, p, i64, i32, i32, i32, p, p, i32]
        lib.oracle_bf.restype = None
        lib.oracle_dist.argtypes = [p, i64, p, i64, i32, i32, p, i32]
        lib.oracle_dist.restype = None
        lib.oracle_bf_lists.argtypes = [p, i64, p, i32, i32, i32, p, p, p, p, i32]
        lib.oracle_bf_lists.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# Brute force primitive (Section 3)
# ---------------------------------------------------------------------------


def bf(Q, X, k: int, metric="l2", threads: int = 0):
    """BF(Q, X): ids [m, k] int64 and rho [m, k] float64, sorted by (rho, id).

    Positions beyond n hold id -1 and rho = +inf.
    """
    Q, X = _f32(Q), _f32(X)
    m, d = Q.shape
    n = X.shape[0]
    assert X.shape[1] == d and k >= 1
    ids = np.empty((m, k), dtype=np.int64)
    rho = np.empty((m, k), dtype=np.float64)
    _load().oracle_bf(_ptr(Q), m, _ptr(X), n, d, k, _METRICS[metric], _ptr(ids), _ptr(rho), threads)
    return ids, rho


def dist(Q, X, metric="l2", threads: int = 0) -> np.ndarray:
    """All rho(q, x) as a float64 [m, n] matrix (small inputs only)."""
    Q, X = _f32(Q), _f32(X)
    out = np.empty((Q.shape[0], X.shape[0]), dtype=np.float64)
    _load().oracle_dist(_ptr(Q), Q.shape[0], _ptr(X), X.shape[0], Q.shape[1], _METRICS[metric], _ptr(out), threads)
    return out


def bf_lists(Q, X, lists, k: int, metric="l2", threads: int = 0):
    """BF(q_i, X[L_i]) for each query i with its own id list ``lists[i]``."""
    Q, X = _f32(Q), _f32(X)
    m, d = Q.shape
    off = np.zeros(m + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    flat = np.ascontiguousarray(
        np.concatenate([np.asarray(l, dtype=np.int64) for l in lists]) if m else np.zeros(0, np.int64)
    )
    ids = np.empty((m, k), dtype=np.int64)
    rho = np.empty((m, k), dtype=np.float64)
    _load().oracle_bf_lists(
        _ptr(Q), m, _ptr(X), d, k, _METRICS[metric], _ptr(off), _ptr(flat), _ptr(ids), _ptr(rho), threads
    )
    return ids, rho


# ---------------------------------------------------------------------------
# Representative sampling (Section 4)
# ---------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state advances by the
    golden-ratio gamma 0x9E3779B97F4A7C15, output is the state passed through
    the variant-13 mixer (shifts 30/27/31)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def below(self, bound: int) -> int:
        """Uniform integer in [0, bound): draws at or above the largest multiple
        of ``bound`` that fits in 2^64 are rejected, so ``x mod bound`` is
        unbiased."""
        limit = (1 << 64) - ((1 << 64) % bound)
        while True:
            x = self.next()
            if x < limit:
                return x % bound


def sample_reps(n: int, n_r: int, seed: int) -> np.ndarray:
    """R: ``n_r`` distinct database ids, uniform without replacement, sorted.

    The paper draws each point independently with probability n_r / n
    (Section 4); the fixed-size reading keeps |R| = n_r exactly.  Step i of a
    partial Fisher-Yates shuffle of [0, n) swaps position i with a uniform
    position in [i, n); the first n_r positions are the sample.  Positions not
    yet touched hold their own index, so a dict stands in for the array.
    """
    assert 1 <= n_r <= n
    g = SplitMix64(seed)
    slot: dict[int, int] = {}
    out = np.empty(n_r, dtype=np.int64)
    for i in range(n_r):
        j = i + g.below(n - i)
        vi, vj = slot.get(i, i), slot.get(j, j)
        slot[i], slot[j] = vj, vi
        out[i] = vj
    out.sort()
    return out


# ---------------------------------------------------------------------------
# Exact RBC (Sections 4 and 5.2)
# ---------------------------------------------------------------------------


@dataclass
class ExactIndex:
    X: np.ndarray  # [n, d] float32 database
    reps: np.ndarray  # [n_r] int64 representative ids, ascending
    owner: np.ndarray  # [n] int64 representative ordinal owning each point
    owner_rho: np.ndarray  # [n] float64 rho(x, owner(x))
    lists: list  # n_r arrays of point ids (ascending)
    psi: np.ndarray  # [n_r] float64 radius max_{x in L_r} rho(x, r); 0 if empty
    metric: str


def build_exact(X, reps, metric="l2", threads: int = 0) -> ExactIndex:
    """Exact-search build: BF(X, R), then each x joins the list of its nearest
    representative, and psi_r = max over the list of rho(x, r) (Sections 4, 5.2).

    Equal distances resolve to the smaller representative id, which is the
    smaller ordinal because R is sorted.
    """
    X = _f32(X)
    reps = np.asarray(reps, dtype=np.int64)
    R = X[reps]
    own, rho = bf(X, R, 1, metric, threads)
    owner = own[:, 0]
    owner_rho = rho[:, 0]
    order = np.argsort(owner, kind="stable")  # ids ascending within each list
    counts = np.bincount(owner, minlength=len(reps))
    bounds = np.concatenate([[0], np.cumsum(counts)])
    lists = [order[bounds[r] : bounds[r + 1]] for r in range(len(reps))]
    psi = np.zeros(len(reps), dtype=np.float64)
    np.maximum.at(psi, owner, owner_rho)
    return ExactIndex(X, reps, owner, owner_rho, lists, psi, metric)


@dataclass
class SearchStats:
    gamma1: np.ndarray  # distance to the nearest representative
    gammak: np.ndarray  # distance to the k-th nearest representative (inf if n_r < k)
    kept: list  # per query: ordinals of the representatives that survive pruning
    examined: np.ndarray  # per query: number of points in the kept lists


def search_exact(index: ExactIndex, Q, k: int, threads: int = 0):
    """Exact search (Section 5.2) generalised to k neighbours.

    1. BF(q, R) keeping every distance D_r = rho(q, r); gamma_1 = min_r D_r and
       gamma_k = the k-th smallest D_r (+inf when n_r < k).
    2. Keep r iff D_r <= gamma_k + psi_r (rule (1), pruning only on strict
       excess) and D_r <= 2 gamma_k + gamma_1 (Lemma 1; 3 gamma at k = 1).
    3. BF(q, X[union of the kept lists]).
    """
    Q = _f32(Q)
    reps = index.reps
    D = dist(Q, index.X[reps], index.metric, threads)
    n_r = len(reps)
    srt = np.sort(D, axis=1)
    g1 = srt[:, 0]
    gk = srt[:, k - 1] if n_r >= k else np.full(Q.shape[0], np.inf)
    keep = (D <= (gk[:, None] + index.psi[None, :])) & (D <= (2.0 * gk + g1)[:, None])
    kept = [np.nonzero(keep[i])[0] for i in range(Q.shape[0])]
    cand = [
        np.sort(np.concatenate([index.lists[r] for r in kr])) if len(kr) else np.zeros(0, np.int64)
        for kr in kept
    ]
    ids, rho = bf_lists(Q, index.X, cand, k, index.metric, threads)
    stats = SearchStats(g1, gk, kept, np.array([len(c) for c in cand], dtype=np.int64))
    return ids, rho, stats


# ---------------------------------------------------------------------------
# One-shot RBC (Sections 4 and 5.1)
# ---------------------------------------------------------------------------


@dataclass
class OneShotIndex:
    X: np.ndarray
    reps: np.ndarray
    lists: np.ndarray  # [n_r, s] ids of the s nearest points of each rep, by (rho, id)
    psi: np.ndarray  # [n_r] the s-th distance
    metric: str


def build_oneshot(X, reps, s: int, metric="l2", threads: int = 0) -> OneShotIndex:
    """One-shot build: BF(R, X) with k = s; L_r is the s nearest database
    points of r (r itself included, rho(r, r) = 0), psi_r their radius."""
    X = _f32(X)
    reps = np.asarray(reps, dtype=np.int64)
    ids, rho = bf(X[reps], X, s, metric, threads)
    return OneShotIndex(X, reps, ids, rho[:, -1].copy(), metric)


def search_oneshot(index: OneShotIndex, Q, k: int, threads: int = 0):
    """One-shot search: r = BF(q, R) (nearest rep, ties to the smaller id),
    then BF(q, X[L_r])."""
    Q = _f32(Q)
    near, _ = bf(Q, index.X[index.reps], 1, index.metric, threads)
    lists = [index.lists[r] for r in near[:, 0]]
    ids, rho = bf_lists(Q, index.X, lists, k, index.metric, threads)
    return ids, rho, near[:, 0]


def rank_of(Q, X, returned_ids, metric="l2", threads: int = 0) -> np.ndarray:
    """Rank error of Section 7.2: number of database points strictly closer to
    q than the returned point (0 = exact nearest neighbour)."""
    Q, X = _f32(Q), _f32(X)
    out = np.empty(len(returned_ids), dtype=np.int64)
    for i, rid in enumerate(returned_ids):
        D = dist(Q[i : i + 1], X, metric, threads)[0]
        out[i] = int(np.count_nonzero(D < D[rid]))
    return out

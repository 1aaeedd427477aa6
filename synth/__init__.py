"""Seeded synthetic inputs for the nearest-neighbour workloads.

This module only draws random numbers; it holds none of the search method's
arithmetic (no distances, no selection, no representatives).  Both the CPU
oracle and the CUDA path (tests, bench) take their inputs from here, so the
two sides see byte-identical float32 arrays.

Generators follow the workload recipes (all float32, row-major [count, d]):

* ``iid_normal``       -- i.i.d. N(0,1) coordinates.
* ``subspace``         -- points on a random k-dim linear subspace of R^d
                          (orthonormal basis from a QR of an N(0,1) matrix,
                          latent coordinates N(0,1)) plus isotropic Gaussian
                          noise of the given *variance*.
* ``clusters``         -- mixture of Gaussian clusters, centres N(0,I), per
                          cluster sigma log-uniform, equal weights.
* ``sincos``           -- a nonlinear embedding [sin(Wz+b), cos(Wz+b)] of a
                          latent N(0,I) vector plus Gaussian noise.
* ``grid``             -- integer lattice points (for closed-form checks).

Seeds: database ``seed``, queries ``seed + 1``; the representative sampler
(seed + 2 by convention) lives with the method, not here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "iid_normal",
    "SubspaceModel",
    "ClusterModel",
    "SincosModel",
    "grid_points",
    "Workload",
    "WORKLOADS",
    "make_workload",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.uint64(seed))


def iid_normal(count: int, d: int, seed: int) -> np.ndarray:
    """[count, d] float32 with i.i.d. N(0,1) entries."""
    return _rng(seed).standard_normal((count, d), dtype=np.float32)


@dataclass
class SubspaceModel:
    """x = A z + e, A: d x k orthonormal columns, z ~ N(0, I_k), e ~ N(0, var I_d)."""

    d: int = 64
    k: int = 8
    noise_var: float = 0.01
    seed: int = 0
    basis: np.ndarray = field(init=False, repr=False)

    def __post_init__(self) -> None:
        g = _rng(self.seed ^ 0x5EED_BA515)
        a = g.standard_normal((self.d, self.k))
        qmat, _ = np.linalg.qr(a)
        self.basis = qmat.astype(np.float64)

    def sample(self, count: int, seed: int, chunk: int = 1 << 18) -> np.ndarray:
        g = _rng(seed)
        out = np.empty((count, self.d), dtype=np.float32)
        sd = math.sqrt(self.noise_var)
        for s in range(0, count, chunk):
            e = min(count, s + chunk)
            z = g.standard_normal((e - s, self.k))
            noise = g.standard_normal((e - s, self.d)) * sd
            out[s:e] = (z @ self.basis.T + noise).astype(np.float32)
        return out


@dataclass
class ClusterModel:
    """Equal-weight mixture of ``n_clusters`` Gaussians in R^d.

    Centres ~ N(0, I_d); sigma_j = exp(U[ln lo, ln hi]); x = mu_j + sigma_j N(0, I).
    """

    d: int = 128
    n_clusters: int = 1000
    sigma_lo: float = 0.05
    sigma_hi: float = 0.5
    seed: int = 0
    centres: np.ndarray = field(init=False, repr=False)
    sigmas: np.ndarray = field(init=False, repr=False)

    def __post_init__(self) -> None:
        g = _rng(self.seed ^ 0xC1_057E25)
        self.centres = g.standard_normal((self.n_clusters, self.d))
        self.sigmas = np.exp(
            g.uniform(math.log(self.sigma_lo), math.log(self.sigma_hi), self.n_clusters)
        )

    def sample(self, count: int, seed: int, chunk: int = 1 << 18) -> np.ndarray:
        g = _rng(seed)
        out = np.empty((count, self.d), dtype=np.float32)
        for s in range(0, count, chunk):
            e = min(count, s + chunk)
            j = g.integers(0, self.n_clusters, e - s)
            noise = g.standard_normal((e - s, self.d))
            out[s:e] = (self.centres[j] + self.sigmas[j, None] * noise).astype(np.float32)
        return out


@dataclass
class SincosModel:
    """x = [sin(W z + b), cos(W z + b)] + N(0, var I); z ~ N(0, I_k), W ~ N(0, 1/k)."""

    d: int = 96
    k: int = 12
    noise_var: float = 0.02
    seed: int = 0
    W: np.ndarray = field(init=False, repr=False)
    b: np.ndarray = field(init=False, repr=False)

    def __post_init__(self) -> None:
        assert self.d % 2 == 0
        g = _rng(self.seed ^ 0x51_7C05)
        self.W = g.standard_normal((self.d // 2, self.k)) / math.sqrt(self.k)
        self.b = g.uniform(0.0, 2.0 * math.pi, self.d // 2)

    def sample(self, count: int, seed: int, chunk: int = 1 << 18) -> np.ndarray:
        g = _rng(seed)
        out = np.empty((count, self.d), dtype=np.float32)
        sd = math.sqrt(self.noise_var)
        h = self.d // 2
        for s in range(0, count, chunk):
            e = min(count, s + chunk)
            z = g.standard_normal((e - s, self.k))
            t = z @ self.W.T + self.b
            noise = g.standard_normal((e - s, self.d)) * sd
            out[s:e, :h] = (np.sin(t) + noise[:, :h]).astype(np.float32)
            out[s:e, h:] = (np.cos(t) + noise[:, h:]).astype(np.float32)
        return out


def grid_points(side: int, d: int) -> np.ndarray:
    """All points of {0, ..., side-1}^d as float32, in lexicographic order."""
    axes = [np.arange(side, dtype=np.float32)] * d
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1).astype(np.float32)


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    m: int
    d: int
    n_r: int
    generator: str
    params: dict


WORKLOADS = {
    # plain N(0,1) database and queries
    "iid-n16k-d16": Workload("iid-n16k-d16", 16384, 1024, 16, 128, "iid", {}),
    # 8-dim linear subspace of R^64 plus N(0, 0.01) noise (variance)
    "subspace8-n1m-d64": Workload(
        "subspace8-n1m-d64", 1 << 20, 100_000, 64, 1024, "subspace", {"k": 8, "noise_var": 0.01}
    ),
    # 1000 Gaussian clusters in R^128
    "clusters1000-n4m-d128": Workload(
        "clusters1000-n4m-d128", 1 << 22, 65_536, 128, 2048, "clusters", {"n_clusters": 1000}
    ),
    # 12-dim nonlinear sin/cos embedding in R^96 plus N(0, 0.02) noise
    "sincos12-n8m-d96": Workload(
        "sincos12-n8m-d96", 1 << 23, 4096, 96, 2896, "sincos", {"k": 12, "noise_var": 0.02}
    ),
}


def make_workload(
    w: Workload | str,
    seed: int = 0,
    n: int | None = None,
    m: int | None = None,
    query_seed: int | None = None,
) -> tuple[np.ndarray, np.ndarray]:
    """(X [n,d], Q [m,d]) float32 for a named workload; ``n``/``m`` override
    sizes; queries use ``query_seed`` (default seed + 1) with the same model."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    n = w.n if n is None else n
    m = w.m if m is None else m
    qs = seed + 1 if query_seed is None else query_seed
    if w.generator == "iid":
        return iid_normal(n, w.d, seed), iid_normal(m, w.d, qs)
    if w.generator == "subspace":
        mod = SubspaceModel(d=w.d, seed=seed, **w.params)
    elif w.generator == "clusters":
        mod = ClusterModel(d=w.d, seed=seed, **w.params)
    elif w.generator == "sincos":
        mod = SincosModel(d=w.d, seed=seed, **w.params)
    else:  # pragma: no cover
        raise ValueError(w.generator)
    return mod.sample(n, seed), mod.sample(m, qs)

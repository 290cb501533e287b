"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on GloVe-100 (1.18 M unit vectors, d = 100), SIFT-128,
GIST-960 and Deep-96 (Section 2 and Table 5).  None of those vectors is
available here, so these generators stand in for them: clustered Gaussian
mixtures (Euclidean), von Mises-Fisher-like mixtures on the unit sphere
(angular, like L2-normalised GloVe) and a uint8 variant of the Gaussian
mixture (like SIFT's byte-valued descriptors).

This module holds input generation only (numpy PCG64 streams); it contains
none of the method's arithmetic, and both the CUDA path's tests and the CPU
oracle's tests draw their inputs from it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def padded_ld(d: int, elsize: int) -> int:
    """Row stride in elements so that every row starts on a 16-byte boundary."""
    per = 16 // elsize
    return (d + per - 1) // per * per


def _pad(X: np.ndarray, ld: int) -> np.ndarray:
    if X.shape[1] == ld:
        return np.ascontiguousarray(X)
    out = np.zeros((X.shape[0], ld), X.dtype)
    out[:, : X.shape[1]] = X
    return out


def equal_sizes(n: int, k: int) -> np.ndarray:
    s = np.full(k, n // k, np.int64)
    s[: n - s.sum()] += 1
    return s


def zipf_sizes(n: int, k: int, s: float = 1.1) -> np.ndarray:
    """Cluster sizes proportional to rank^-s, made integral by largest remainder."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    q = w / w.sum() * n
    base = np.floor(q).astype(np.int64)
    rem = n - int(base.sum())
    order = np.argsort(-(q - base), kind="stable")
    base[order[:rem]] += 1
    return base


def _labels(sizes: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    lab = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
    rng.shuffle(lab)
    return lab


@dataclass
class PointSet:
    X: np.ndarray            # (n, ld) float32 or uint8, zero padded beyond d
    d: int
    metric: int              # 0 = L2 f32, 1 = angular f32, 2 = L2 u8
    labels: np.ndarray       # cluster of each point
    centres: np.ndarray      # (k, d) float64
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def ld(self) -> int:
        return self.X.shape[1]


def gaussian_mixture(n: int, d: int, k: int, seed: int, centre_std: float = 5.0,
                     sigma: float = 1.0) -> PointSet:
    """Isotropic mixture: centres ~ N(0, centre_std^2 I), points = centre + N(0, sigma^2 I),
    equal cluster sizes, ids in shuffled order."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, centre_std, size=(k, d))
    lab = _labels(equal_sizes(n, k), rng)
    X = centres[lab] + rng.normal(0.0, sigma, size=(n, d))
    return PointSet(_pad(X.astype(np.float32), padded_ld(d, 4)), d, 0, lab, centres,
                    dict(kind="gauss", k=k, seed=seed, centre_std=centre_std, sigma=sigma))


def gaussian_queries(ps: PointSet, nq: int, seed: int) -> np.ndarray:
    """Held-out queries from the same centres, drawn from the stream seed."""
    rng = np.random.default_rng(seed)
    k = ps.centres.shape[0]
    lab = rng.integers(0, k, size=nq)
    Q = ps.centres[lab] + rng.normal(0.0, ps.meta["sigma"], size=(nq, ps.d))
    return _pad(Q.astype(np.float32), ps.ld)


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def vmf_like(n: int, d: int, k: int, seed: int, kappa: float = 20.0,
             sizes: str = "equal", zipf_s: float = 1.1) -> PointSet:
    """Unit vectors x = normalise(mu_c + g / sqrt(kappa)), mu_c uniform on the sphere,
    g ~ N(0, I); cluster sizes equal or Zipf(zipf_s)."""
    rng = np.random.default_rng(seed)
    mu = _unit(rng.normal(size=(k, d)))
    sz = equal_sizes(n, k) if sizes == "equal" else zipf_sizes(n, k, zipf_s)
    lab = _labels(sz, rng)
    X = np.empty((n, d), np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        g = rng.normal(size=(e - s, d))
        X[s:e] = _unit(mu[lab[s:e]] + g / math.sqrt(kappa)).astype(np.float32)
    return PointSet(_pad(X, padded_ld(d, 4)), d, 1, lab, mu,
                    dict(kind="vmf", k=k, seed=seed, kappa=kappa, sizes=sizes))


def vmf_queries(ps: PointSet, nq: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    k = ps.centres.shape[0]
    lab = rng.integers(0, k, size=nq)
    g = rng.normal(size=(nq, ps.d))
    Q = _unit(ps.centres[lab] + g / math.sqrt(ps.meta["kappa"])).astype(np.float32)
    return _pad(Q, ps.ld)


def _to_u8(z: np.ndarray, var: float) -> np.ndarray:
    return np.clip(np.rint(60.0 + 30.0 * z / math.sqrt(var)), 0, 255).astype(np.uint8)


def uint8_mixture(n: int, d: int, k: int, seed: int) -> PointSet:
    """Byte vectors x = clip(round(60 + 30 z / sqrt(26)), 0, 255) with z drawn from the
    Gaussian mixture above (per-coordinate variance 25 + 1 = 26)."""
    g = gaussian_mixture(n, d, k, seed)
    z = g.X[:, :d].astype(np.float64)
    X = _to_u8(z, 26.0)
    return PointSet(_pad(X, padded_ld(d, 1)), d, 2, g.labels, g.centres,
                    dict(kind="u8", k=k, seed=seed, sigma=1.0))


def uint8_queries(ps: PointSet, nq: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    k = ps.centres.shape[0]
    lab = rng.integers(0, k, size=nq)
    z = ps.centres[lab] + rng.normal(0.0, 1.0, size=(nq, ps.d))
    return _pad(_to_u8(z, 26.0), ps.ld)


def queries(ps: PointSet, nq: int, seed: int) -> np.ndarray:
    if ps.meta["kind"] == "vmf":
        return vmf_queries(ps, nq, seed)
    if ps.meta["kind"] == "u8":
        return uint8_queries(ps, nq, seed)
    return gaussian_queries(ps, nq, seed)


def intra_cluster_blocks(labels: np.ndarray, n_blocks: int, bs: int, seed: int) -> np.ndarray:
    """n_blocks blocks of bs ids, each sampled without replacement from one cluster;
    clusters smaller than bs are skipped; clusters are visited round-robin."""
    rng = np.random.default_rng(seed)
    k = int(labels.max()) + 1
    members = [np.flatnonzero(labels == c).astype(np.int32) for c in range(k)]
    big = [m for m in members if len(m) >= bs]
    if not big:
        raise ValueError("no cluster holds a full block")
    out = np.empty((n_blocks, bs), np.int32)
    for b in range(n_blocks):
        m = big[b % len(big)]
        out[b] = np.sort(rng.choice(m, size=bs, replace=False))
    return out


# The five workloads, by what they are.  Parameters follow the paper's shapes:
# T trees, R degree bound, ef_h harvest width, alpha prune factor, B blocks.
WORKLOADS = {
    "tiny-gauss-n2000-d16": dict(gen="gauss", n=2000, d=16, k=8, T=4, R=16, ef_h=32,
                                 alpha=1.2, B=(1, 4), nq=200, seed=0),
    "incache-angular-n100k-d100": dict(gen="vmf", n=100_000, d=100, k=64, kappa=20.0,
                                       sizes="equal", T=8, R=32, ef_h=64, alpha=1.2, B=(8,),
                                       nq=10_000, seed=0),
    "paper-angular-n1183514-d100": dict(gen="vmf", n=1_183_514, d=100, k=256, kappa=20.0,
                                        sizes="zipf", T=8, R=64, ef_h=100, alpha=1.2,
                                        B=(1, 2, 4, 8, 16), nq=10_000, seed=0),
}


def make_points(spec: dict, n: int | None = None, d: int | None = None) -> PointSet:
    n = spec["n"] if n is None else n
    d = spec["d"] if d is None else d
    if spec["gen"] == "gauss":
        return gaussian_mixture(n, d, spec["k"], spec["seed"])
    if spec["gen"] == "vmf":
        return vmf_like(n, d, spec["k"], spec["seed"], spec.get("kappa", 20.0),
                        spec.get("sizes", "equal"))
    if spec["gen"] == "u8":
        return uint8_mixture(n, d, spec["k"], spec["seed"])
    raise ValueError(spec["gen"])

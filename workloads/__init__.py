"""Seeded synthetic two-table inputs shared by the tests, the bench and smoke().

This module holds no part of the method's arithmetic: it only draws tables
(features + int32 join keys) with the shapes and distributions of the
paper's workloads (synthetic relations, Section 2) and of the five
benchmark configurations:

* ``c0``  1,000 + 1,000 rows, 4 + 4 FP64 features U[-1,1], 100 keys.
* ``c1``  1e6 + 1e6 rows, 16 + 16 FP32 features N(0,1), 10,000 keys.
* ``c2``  4e6 + 2e6 rows, 32 + 32 FP32 features U[-1,1], Zipf(1.2) keys over
          1e5 ids (a seeded permutation of the rank, so hot keys are not the
          small integers).
* ``c3``  512 instances, m1, m2 log-uniform in [1e3, 1e5], n1, n2 from
          {8, 16, 32, 64}, FP32 N(0,1), K = max(1, min(m1, m2) // 10) keys.
* ``c4``  2e5 + 2e5 rows, 256 + 256 FP32 features; A N(0,1), B = B0 * D with
          D_jj = 10^(-8 j / (n2 - 1)) (column scaling, condition 1e8), 100 keys.
* ``c4_stress``  c4 with truly ill-conditioned B = B0 V D V^T, V a random
          (Haar) orthogonal matrix: the small singular directions are not
          columns, so no column scaling undoes them (condition 1e8).
* ``paper_shape``  the paper's own experiment: one key (Cartesian product),
          m rows per table, U(0,1) features.

Tables are drawn i.i.d. row by row: they are not pre-sorted by key.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 0x250323385


@dataclasses.dataclass
class Table:
    x: np.ndarray    # (m, n) row-major features, float32 or float64
    key: np.ndarray  # (m,) int32 join keys

    @property
    def m(self) -> int:
        return int(self.x.shape[0])

    @property
    def n(self) -> int:
        return int(self.x.shape[1])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _features(rng, m, n, dist, dtype):
    if dist == "uniform_pm1":
        x = rng.uniform(-1.0, 1.0, size=(m, n))
    elif dist == "uniform01":
        x = rng.uniform(0.0, 1.0, size=(m, n))
    elif dist == "normal":
        x = rng.standard_normal(size=(m, n))
    else:
        raise ValueError(dist)
    return np.ascontiguousarray(x.astype(dtype))


def uniform_keys(rng, m, num_keys, offset=0):
    return (rng.integers(0, max(int(num_keys), 1), size=m, dtype=np.int64) + offset).astype(np.int32)


def zipf_keys(rng, m, num_keys, s, ids):
    """Keys whose rank r = 1..num_keys has probability proportional to r^-s,
    by inverse-CDF search; the rank is mapped through the id permutation."""
    w = np.arange(1, num_keys + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(m)
    rank = np.minimum(np.searchsorted(cdf, u, side="right"), num_keys - 1)
    return ids[rank].astype(np.int32)


def random_orthogonal(rng, n):
    """A Haar-distributed n x n orthogonal matrix: the orthogonal factor of a
    Gaussian matrix with its columns' signs fixed (Mezzadri, Notices AMS 2007)."""
    q, r = np.linalg.qr(rng.standard_normal(size=(n, n)))
    return q * np.sign(np.diag(r))


def make_pair(m1, n1, m2, n2, num_keys, dtype=np.float32, dist="normal", seed=0, key_offset=0):
    """Two tables with uniform keys over [key_offset, key_offset + num_keys)."""
    ra, rb = _rng(seed * 2 + 1), _rng(seed * 2 + 2)
    A = Table(_features(ra, m1, n1, dist, dtype), uniform_keys(ra, m1, num_keys, key_offset))
    B = Table(_features(rb, m2, n2, dist, dtype), uniform_keys(rb, m2, num_keys, key_offset))
    return A, B


def config(name: str, scale: float = 1.0, rank: int = 0):
    """Tables of a named configuration.  ``scale`` < 1 shrinks the row counts
    (and key counts in proportion) for quick runs; ``rank`` selects an
    independent replica (different seed) for multi-process runs."""
    cfg = {"c0": 0, "c1": 1, "c2": 2, "c3": 3, "c4": 4, "paper_shape": 5, "c4_stress": 4}[name]
    seed = BASE_SEED + 1000 * cfg + 100000 * rank

    def rows(v):
        return max(1, int(round(v * scale)))

    if name == "c0":
        return make_pair(rows(1000), 4, rows(1000), 4, max(1, rows(100)), np.float64, "uniform_pm1", seed)
    if name == "c1":
        return make_pair(rows(1_000_000), 16, rows(1_000_000), 16, max(1, rows(10_000)), np.float32, "normal", seed)
    if name == "c2":
        nk = max(1, rows(100_000))
        ids = _rng(seed + 7).permutation(nk).astype(np.int64)
        ra, rb = _rng(seed + 1), _rng(seed + 2)
        m1, m2 = rows(4_000_000), rows(2_000_000)
        A = Table(_features(ra, m1, 32, "uniform_pm1", np.float32), zipf_keys(ra, m1, nk, 1.2, ids))
        B = Table(_features(rb, m2, 32, "uniform_pm1", np.float32), zipf_keys(rb, m2, nk, 1.2, ids))
        return A, B
    if name in ("c4", "c4_stress"):
        nk = 100
        ra, rb = _rng(seed + 1), _rng(seed + 2)
        m = rows(200_000)
        A = Table(_features(ra, m, 256, "normal", np.float32), uniform_keys(ra, m, nk))
        b0 = rb.standard_normal(size=(m, 256))
        d = 10.0 ** (-8.0 * np.arange(256) / 255.0)
        if name == "c4":
            b = b0 * d
        else:
            v = random_orthogonal(_rng(seed + 9), 256)
            b = b0 @ (v * d) @ v.T
        B = Table(np.ascontiguousarray(b.astype(np.float32)), uniform_keys(rb, m, nk))
        return A, B
    if name == "paper_shape":
        m = rows(1600)
        ra, rb = _rng(seed + 1), _rng(seed + 2)
        A = Table(_features(ra, m, 32, "uniform01", np.float32), np.zeros(m, np.int32))
        B = Table(_features(rb, m, 32, "uniform01", np.float32), np.zeros(m, np.int32))
        return A, B
    if name == "c3":
        return batch_instances(count=max(1, rows(512)), seed=seed)
    raise ValueError(name)


def batch_instances(count=512, seed=BASE_SEED + 3000, lo=1e3, hi=1e5, widths=(8, 16, 32, 64), max_rows=None):
    """Independent instances: m1, m2 log-uniform in [lo, hi], n1, n2 uniform
    over ``widths``, FP32 N(0,1), keys uniform over max(1, min(m1, m2)//10)."""
    meta = _rng(seed)
    out = []
    for i in range(count):
        m1 = int(round(math.exp(meta.uniform(math.log(lo), math.log(hi)))))
        m2 = int(round(math.exp(meta.uniform(math.log(lo), math.log(hi)))))
        if max_rows is not None:
            m1, m2 = min(m1, max_rows), min(m2, max_rows)
        n1 = int(meta.choice(widths))
        n2 = int(meta.choice(widths))
        K = max(1, min(m1, m2) // 10)
        out.append(make_pair(m1, n1, m2, n2, K, np.float32, "normal", seed * 7 + i))
    return out

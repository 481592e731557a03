"""Seeded synthetic inputs shaped like the paper's low-rank matrix workloads.

This module only draws random numbers and assembles problem data (sparse
patterns, sampled entries, graph Laplacian cost matrices, random start
blocks).  It holds none of the polynomial-filtered method's arithmetic, so the
CPU oracle and the CUDA path can both take their inputs from here without
sharing any of the computation they are compared on.

Workload laws:

* PSD matrix completion (the symmetric analogue of the matrix-completion
  tests of Sec. 5.2, Example "MC"): ``M = G G^T`` with ``G`` an ``n x r``
  Gaussian matrix of variance ``1/r``; the sample set Omega draws each
  unordered pair ``i <= j`` independently with probability ``rate`` and is
  mirrored, so the stored pattern is symmetric.  Sampled values are stored in
  float32 (CSR, int32 column indices, sorted columns).
* Max-cut SDP (a standard SDP, Sec. 2.3): an Erdos-Renyi graph with edge
  probability ``prob``, no self loops, weights +-1 with equal probability,
  and cost matrix ``C = -L/4`` with ``L = D - W`` the weighted Laplacian,
  stored as a CSR matrix that includes the diagonal.
* Matrix completion for SVT (Example "MC" of Sec. 5.2): ``M = M_L M_R^T``
  with standard Gaussian ``n x r`` factors; every entry is observed
  independently with probability ``SR`` (Bernoulli sampling standing in for
  a uniform draw of exactly ``SR n^2`` pairs).  The pattern is stored twice:
  row-major CSR, and the CSR of the transpose with the permutation that maps
  its entries to the row-major ones (an input format, like CSR itself).
* Start block: an ``n x p`` standard Gaussian matrix.  Orthonormalising it
  is the method's job, not the generator's.

Seeds: ``seed = 1904105850 + config_index`` with numpy ``PCG64``; the
graph/weights, the sample set, the factor ``G`` and the start block draw from
independent child streams made by ``SeedSequence.spawn``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1904105850


def config_seed(config_index: int) -> int:
    return SEED_BASE + int(config_index)


def _streams(seed: int, k: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(k)]


@dataclasses.dataclass
class CSR:
    """Square sparse matrix in CSR form (int32 indices, sorted columns)."""

    n: int
    rowptr: np.ndarray  # int32 [n+1]
    colind: np.ndarray  # int32 [nnz]
    vals: np.ndarray    # float32 or float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        a[rows, self.colind] = self.vals.astype(np.float64)
        return a

    def row_of_entries(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.rowptr))


def _upper_pairs(rng, n: int, prob: float, include_diag: bool):
    """Independent Bernoulli(prob) draw over the unordered pairs i <= j
    (i < j when ``include_diag`` is False), by geometric skips over the
    row-major enumeration of the upper triangle.  Returns sorted (i, j)."""
    if n <= 0 or prob <= 0.0:
        e = np.zeros(0, dtype=np.int64)
        return e, e
    width = n if include_diag else n - 1
    # row i holds columns j = i + (0 if include_diag else 1) .. n-1
    counts = np.arange(width, 0, -1, dtype=np.int64) if include_diag else np.arange(n - 1, 0, -1, dtype=np.int64)
    total = int(counts.sum())
    if total == 0:
        e = np.zeros(0, dtype=np.int64)
        return e, e
    if prob >= 1.0:
        lin = np.arange(total, dtype=np.int64)
    else:
        # expected count plus a generous margin; top up if ever short
        est = int(total * prob + 10 * math.sqrt(total * prob + 1) + 16)
        chunks = []
        pos = -1
        while True:
            gaps = rng.geometric(prob, size=est).astype(np.int64)
            cs = pos + np.cumsum(gaps)
            chunks.append(cs[cs < total])
            if cs[-1] >= total:
                break
            pos = int(cs[-1])
        lin = np.concatenate(chunks)
    offsets = np.concatenate([[0], np.cumsum(counts)])
    i = np.searchsorted(offsets, lin, side="right") - 1
    start = i + (0 if include_diag else 1)
    j = start + (lin - offsets[i])
    return i.astype(np.int64), j.astype(np.int64)


def _symmetric_csr(n: int, i: np.ndarray, j: np.ndarray, v: np.ndarray, diag=None) -> CSR:
    """Mirror upper-triangle entries (i <= j) into a full symmetric CSR."""
    off = i != j
    rows = np.concatenate([i, j[off]])
    cols = np.concatenate([j, i[off]])
    vals = np.concatenate([v, v[off]])
    if diag is not None:
        rows = np.concatenate([rows, np.arange(n)])
        cols = np.concatenate([cols, np.arange(n)])
        vals = np.concatenate([vals, diag])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    if rowptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 row pointers")
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals)


@dataclasses.dataclass
class CompletionInstance:
    n: int
    rank: int
    G: np.ndarray       # n x rank float64 ground-truth factor, M = G G^T
    omega: CSR          # sampled entries of M (float32 values), symmetric pattern
    U0_raw: np.ndarray  # n x p standard Gaussian start block (not orthonormal)
    mu: float
    t: float


def completion_instance(n: int, rank: int, rate: float, p: int, seed: int,
                        mu: float = 0.05, t: float = 1.0) -> CompletionInstance:
    """PSD completion data: M = G G^T, G ~ N(0, 1/rank); Omega symmetric
    uniform with pair probability ``rate`` (diagonal pairs included)."""
    r_pat, r_g, r_u = _streams(seed, 3)
    G = r_g.standard_normal((n, rank)) / math.sqrt(rank)
    i, j = _upper_pairs(r_pat, n, rate, include_diag=True)
    vals = np.empty(i.shape[0], dtype=np.float64)
    step = 1 << 20
    for s in range(0, i.shape[0], step):
        vals[s:s + step] = np.einsum("ij,ij->i", G[i[s:s + step]], G[j[s:s + step]])
    omega = _symmetric_csr(n, i, j, vals.astype(np.float32))
    U0 = r_u.standard_normal((n, p))
    return CompletionInstance(n, rank, G, omega, U0, float(mu), float(t))


@dataclasses.dataclass
class SVTInstance:
    n: int
    rank: int
    ML: np.ndarray          # n x r
    MR: np.ndarray          # n x r
    omega: CSR              # observed entries of M (float64 values), row-major
    t_rowptr: np.ndarray    # CSR of the transpose of the pattern
    t_colind: np.ndarray
    t_perm: np.ndarray      # int32: entry e of the transpose is entry t_perm[e] of omega
    U0_raw: np.ndarray      # n x p standard Gaussian start block


def svt_instance(n: int, rank: int, sr: float, p: int, seed: int) -> SVTInstance:
    r_pat, r_l, r_r, r_u = _streams(seed, 4)
    ML = r_l.standard_normal((n, rank))
    MR = r_r.standard_normal((n, rank))
    rows, cols = [], []
    for i0 in range(0, n, 1024):
        i1 = min(n, i0 + 1024)
        mask = r_pat.random((i1 - i0, n)) < sr
        ii, jj = np.nonzero(mask)
        rows.append((ii + i0).astype(np.int64))
        cols.append(jj.astype(np.int64))
    i = np.concatenate(rows)
    j = np.concatenate(cols)
    vals = np.empty(i.shape[0], dtype=np.float64)
    step = 1 << 20
    for s0 in range(0, i.shape[0], step):
        vals[s0:s0 + step] = np.einsum("ij,ij->i", ML[i[s0:s0 + step]], MR[j[s0:s0 + step]])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, i + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    omega = CSR(n, rowptr, j.astype(np.int32), vals)
    order = np.lexsort((i, j))                    # by column, then row
    t_rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(t_rowptr, j + 1, 1)
    t_rowptr = np.cumsum(t_rowptr).astype(np.int32)
    return SVTInstance(n, rank, ML, MR, omega, t_rowptr, i[order].astype(np.int32),
                       order.astype(np.int32), r_u.standard_normal((n, p)))


@dataclasses.dataclass
class MaxCutInstance:
    n: int
    C: CSR              # C = -L/4 (float64 values), diagonal included
    n_edges: int
    U0_raw: np.ndarray  # n x p standard Gaussian start block


@dataclasses.dataclass
class NCEInstance:
    n: int
    G: np.ndarray       # symmetric test matrix (Sec. 5.1 examples)
    U0_raw: np.ndarray  # n x p standard Gaussian start block


def maxcut_cost_from_edges(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray) -> CSR:
    """C = -(D - W)/4 for the weighted graph with edges (i<j, w)."""
    deg = np.zeros(n, dtype=np.float64)
    np.add.at(deg, i, w)
    np.add.at(deg, j, w)
    return _symmetric_csr(n, i, j, 0.25 * w.astype(np.float64), diag=-0.25 * deg)


def maxcut_instance(n: int, prob: float, p: int, seed: int) -> MaxCutInstance:
    """Erdos-Renyi graph G(n, prob), weights +-1 equiprobable, C = -L/4."""
    r_graph, r_w, r_u = _streams(seed, 3)
    i, j = _upper_pairs(r_graph, n, prob, include_diag=False)
    w = np.where(r_w.random(i.shape[0]) < 0.5, -1.0, 1.0)
    C = maxcut_cost_from_edges(n, i, j, w)
    U0 = r_u.standard_normal((n, p))
    return MaxCutInstance(n, C, int(i.shape[0]), U0)


def dense_symmetric_with_spectrum(n: int, eigvals: np.ndarray, seed: int):
    """B = Q diag(eigvals) Q^T with Q a product of seeded Householder
    reflections (test matrices of known spectrum).  Returns (B, Q)."""
    rng = _streams(seed, 1)[0]
    Q = np.eye(n)
    for _ in range(3):
        v = rng.standard_normal(n)
        v /= np.linalg.norm(v)
        Q = Q - 2.0 * np.outer(Q @ v, v)
    B = (Q * np.asarray(eigvals, dtype=np.float64)) @ Q.T
    B = 0.5 * (B + B.T)
    return B, Q


def gaussian_block(n: int, p: int, seed: int) -> np.ndarray:
    return _streams(seed, 1)[0].standard_normal((n, p))


# Named workloads (sizes of the configurations the benchmark and tests use).
# ``iters`` is the configured iteration count (fixed-count parity runs);
# ``max_iters``, where given, caps a solve that runs to its tolerance.
WORKLOADS = {
    "completion_n400": dict(kind="completion", n=400, rank=8, rate=0.20, p=16, degree=3,
                            iters=100, max_iters=3000, mu=0.05, t=1.0, config_index=0),
    "maxcut_n4096": dict(kind="maxcut", n=4096, prob=0.01, p=32, degree=4, iters=200,
                         max_iters=6000, config_index=1),
    "maxcut_n4096_structured": dict(kind="maxcut", n=4096, prob=0.01, p=32, degree=4, iters=200,
                                    max_iters=6000, config_index=1),
    "maxcut_n16384_lowprec": dict(kind="maxcut", n=16384, prob=0.01, p=64, degree=4,
                                  degree_max=8, iters=200, config_index=2),
    "nce_n4000": dict(kind="nce", n=4000, example="5.7", p=64, degree=3, iters=1000,
                      accel_l=2, config_index=5),
    "completion_n50000": dict(kind="completion", n=50000, rank=20, rate=0.01, p=40, degree=4,
                              iters=100, max_iters=3000, mu=0.05, t=1.0, config_index=3),
    "svt_n5000": dict(kind="svt", n=5000, rank=10, sr=0.1, p=32, degree=1, iters=500,
                      config_index=6),
    "nnls_n10000": dict(kind="nnls", n=10000, rank=10, sr=0.05, p=32, degree=1, iters=300,
                        mu_bar_rel=1e-2, config_index=7),
}


def make_workload(name: str, **overrides):
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    seed = config_seed(cfg["config_index"])
    if cfg["kind"] == "nce":
        rng_u = _streams(seed + 1, 1)[0]
        return cfg, NCEInstance(cfg["n"], nce_matrix(cfg["n"], cfg["example"], seed),
                                rng_u.standard_normal((cfg["n"], cfg["p"])))
    if cfg["kind"] in ("svt", "nnls"):
        return cfg, svt_instance(cfg["n"], cfg["rank"], cfg["sr"], cfg["p"], seed)
    if cfg["kind"] == "completion":
        return cfg, completion_instance(cfg["n"], cfg["rank"], cfg["rate"], cfg["p"], seed,
                                        mu=cfg["mu"], t=cfg["t"])
    return cfg, maxcut_instance(cfg["n"], cfg["prob"], cfg["p"], seed)


def serving_mix(n_requests: int, seed: int, p: int = 32,
                maxcut_n=(512, 8192), completion_n=(2000, 50000), rank=(5, 20),
                rate=(0.01, 0.10), maxcut_prob=0.01):
    """Mixed request stream: half max-cut SDPs (n log-uniform in maxcut_n,
    G(n, maxcut_prob) with +-1 weights), half PSD completions (n log-uniform
    in completion_n, rank uniform in `rank`, sampling rate uniform in `rate`),
    in a seeded random order.  Returns a list of dicts (kind, n, instance)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = ["maxcut"] * (n_requests // 2) + ["completion"] * (n_requests - n_requests // 2)
    rng.shuffle(kinds)
    out = []
    for i, kind in enumerate(kinds):
        sub = int(rng.integers(0, 2**31 - 1))
        if kind == "maxcut":
            lo, hi = maxcut_n
            n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
            n = max(n, p + 1)
            out.append(dict(kind=kind, n=n, inst=maxcut_instance(n, maxcut_prob, p, sub)))
        else:
            lo, hi = completion_n
            n = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
            n = max(n, p + 1)
            r = int(rng.integers(rank[0], rank[1] + 1))
            rt = float(rng.uniform(rate[0], rate[1]))
            out.append(dict(kind=kind, n=n, rank=r, rate=rt,
                            inst=completion_instance(n, r, rt, p, sub)))
    return out


def poisson_arrivals(n_requests: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if rate_per_s <= 0 or not math.isfinite(rate_per_s):
        return np.zeros(n_requests)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n_requests))


def nce_matrix(n: int, example: str, seed: int) -> np.ndarray:
    """Symmetric test matrices of the nearest-correlation examples (Sec. 5.1):
    "5.6": off-diagonal entries uniform in [-1, 1], unit diagonal;
    "5.7": off-diagonal entries uniform in [0, 2], unit diagonal."""
    rng = _streams(seed, 1)[0]
    lo, hi = {"5.6": (-1.0, 1.0), "5.7": (0.0, 2.0)}[example]
    A = rng.uniform(lo, hi, (n, n))
    A = np.triu(A, 1)
    A = A + A.T
    np.fill_diagonal(A, 1.0)
    return A

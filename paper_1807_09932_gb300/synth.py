"""Seeded synthetic inputs shaped like the paper's workloads (arXiv 1807.09932, Table 1).

The GEO datasets the paper runs on (GDS1490, GSE65194, GSE84493) are not available, so every
matrix here is synthetic: a N(0,1) or Beta(0.5, 0.5) background with planted trend biclusters
and uniformly injected NaN. This module holds input generation only -- none of the method's
arithmetic -- and is the one module both the CUDA path's callers and the oracle's tests use.

Recipe (all draws from numpy's PCG64, seeded):
  * background: N(0,1), or Beta(0.5,0.5) drawn as sin^2(pi*U/2) (the arcsine inverse CDF);
  * planted biclusters: row-disjoint row blocks (slices of one random row permutation), columns
    drawn without replacement; in each planted row the values of the planted columns are
    re-ordered to increase (decrease for a negative-trend bicluster) along a random order of
    those columns;
  * NaN: a uniform fraction of all cells, injected after planting (a planted row can lose its
    membership when exclusion is on);
  * populations: candidates with length uniform in [lmin, lmax] (capped at C) and distinct
    columns in random order, stored as CSR (uint16 columns, uint32 offsets, offsets[0] = 0).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 1807099320


@dataclasses.dataclass
class Planted:
    rows: np.ndarray      # int64 row indices (sorted)
    cols: np.ndarray      # column order along which the values follow the trend
    negative: bool        # True: values decrease along ``cols``


@dataclasses.dataclass
class Dataset:
    X: np.ndarray                 # float32 [R, C], C-contiguous
    planted: list
    exclude_missing: bool
    negative: bool                # the request-level negative-trend option for this workload


def background(rng, rows, cols, kind="normal"):
    if kind == "normal":
        return rng.standard_normal((rows, cols), dtype=np.float32)
    if kind == "beta":
        u = rng.random((rows, cols), dtype=np.float32)
        return (np.sin(np.float32(math.pi / 2) * u) ** 2).astype(np.float32)
    raise ValueError(kind)


def plant(rng, X, specs):
    """Plant row-disjoint trend biclusters. ``specs``: list of (n_rows, n_cols, negative)."""
    R, C = X.shape
    perm = rng.permutation(R)
    total = sum(s[0] for s in specs)
    scale = min(1.0, R / max(total, 1))
    out, start = [], 0
    for n_rows, n_cols, negative in specs:
        n_rows = max(1, int(n_rows * scale))
        n_cols = min(n_cols, C)
        rows = np.sort(perm[start:start + n_rows])
        start += n_rows
        order = rng.choice(C, size=n_cols, replace=False)
        block = X[np.ix_(rows, order)]
        block = np.sort(block, axis=1)
        if negative:
            block = block[:, ::-1]
        X[np.ix_(rows, order)] = block
        out.append(Planted(rows=rows.astype(np.int64), cols=order.astype(np.int64),
                           negative=bool(negative)))
    return out


def inject_nan(rng, X, frac):
    if frac <= 0:
        return
    mask = rng.random(X.shape) < frac
    X[mask] = np.nan


def make_dataset(seed, rows, cols, *, kind="normal", planted=(), nan_frac=0.0,
                 exclude_missing=True, negative=False):
    rng = np.random.default_rng(seed)
    X = background(rng, rows, cols, kind)
    pl = plant(rng, X, list(planted))
    inject_nan(rng, X, nan_frac)
    return Dataset(X=np.ascontiguousarray(X), planted=pl, exclude_missing=exclude_missing,
                   negative=negative)


def make_population(seed, n_cand, n_cols, lmin, lmax):
    """Uniform random candidates in CSR form (uint16 cols, uint32 offsets)."""
    rng = np.random.default_rng(seed)
    lmax = min(lmax, n_cols)
    lmin = min(lmin, lmax)
    lengths = rng.integers(lmin, lmax + 1, size=n_cand)
    offsets = np.zeros(n_cand + 1, dtype=np.uint32)
    offsets[1:] = np.cumsum(lengths)
    cols = np.empty(int(offsets[-1]), dtype=np.uint16)
    for i, L in enumerate(lengths):
        cols[offsets[i]:offsets[i + 1]] = rng.choice(n_cols, size=int(L), replace=False)
    return cols, offsets


def population_from_lists(cands):
    """CSR form of a list of column lists."""
    offsets = np.zeros(len(cands) + 1, dtype=np.uint32)
    offsets[1:] = np.cumsum([len(c) for c in cands])
    cols = np.array([c for cand in cands for c in cand], dtype=np.uint16)
    return cols, offsets


def random_bitmaps(seed, n, rows, density=0.3):
    """Random row bitmaps (LSB-first uint32 words, padding bits cleared) for archive inputs."""
    rng = np.random.default_rng(seed)
    bits = rng.random((n, rows)) < density
    W = (rows + 31) // 32
    padded = np.zeros((n, W * 32), dtype=np.uint8)
    padded[:, :rows] = bits
    packed = np.packbits(padded, axis=1, bitorder="little")        # [n, 4W] bytes
    return np.ascontiguousarray(packed).view("<u4").astype(np.uint32).reshape(n, W)


# ---- the five workloads (shapes from the paper's Table 1 and its big-data section) ----------

def config1(seed=BASE_SEED + 1):
    """Small: 1,000 x 50 N(0,1), 3 planted increasing 50 x 8, no NaN; 200 candidates of 2-10."""
    ds = make_dataset(seed, 1000, 50, kind="normal", planted=[(50, 8, False)] * 3,
                      nan_frac=0.0, exclude_missing=True, negative=False)
    cols, offs = make_population(seed + 1000, 200, 50, 2, 10)
    return ds, cols, offs


def config2(seed=BASE_SEED + 2):
    """Expression-shaped: 20,000 x 200 N(0,1), 5 planted (200-2,000 x 6-20, two negative),
    1% NaN with exclusion on, negative option on; 1,600 candidates of 2-20."""
    rng = np.random.default_rng(seed + 7)
    specs = [(int(rng.integers(200, 2001)), int(rng.integers(6, 21)), i < 2) for i in range(5)]
    ds = make_dataset(seed, 20000, 200, kind="normal", planted=specs, nan_frac=0.01,
                      exclude_missing=True, negative=True)
    cols, offs = make_population(seed + 1000, 1600, 200, 2, 20)
    return ds, cols, offs


def config3(seed=BASE_SEED + 3, rows=436444):
    """Methylation-shaped: 436,444 x 64 Beta(0.5,0.5), 10 planted (5,000-50,000 x 5-16),
    0.5% NaN with exclusion on; 1,600 candidates of 2-16."""
    rng = np.random.default_rng(seed + 7)
    specs = [(int(rng.integers(5000, 50001)), int(rng.integers(5, 17)), False)
             for _ in range(10)]
    ds = make_dataset(seed, rows, 64, kind="beta", planted=specs, nan_frac=0.005,
                      exclude_missing=True, negative=False)
    cols, offs = make_population(seed + 1000, 1600, 64, 2, 16)
    return ds, cols, offs


def config4_specs(seed=BASE_SEED + 4):
    """Batched: 8 datasets (rows log-uniform in [5k, 200k], cols uniform in [20, 500], N(0,1) and
    Beta alternating) and 64 populations (sizes uniform in [200, 3,200], lengths 2-64),
    round-robin over the datasets. Returns (dataset specs, population specs)."""
    rng = np.random.default_rng(seed)
    datasets = []
    for d in range(8):
        rows = int(round(math.exp(rng.uniform(math.log(5000), math.log(200000)))))
        cols = int(rng.integers(20, 501))
        datasets.append(dict(seed=seed + 100 + d, rows=rows, cols=cols,
                             kind="normal" if d % 2 == 0 else "beta"))
    pops = []
    for p in range(64):
        pops.append(dict(seed=seed + 10000 + p, dataset=p % 8,
                         n_cand=int(rng.integers(200, 3201)), lmin=2, lmax=64))
    return datasets, pops


def config5_specs(seed=BASE_SEED + 5, n_runs=32):
    """Served: 32 EBIC runs on datasets of 10,000-436,444 rows (log-uniform) x 20-200 cols;
    1,600 candidates per request."""
    rng = np.random.default_rng(seed)
    runs = []
    for i in range(n_runs):
        rows = int(round(math.exp(rng.uniform(math.log(10000), math.log(436444)))))
        cols = int(rng.integers(20, 201))
        runs.append(dict(seed=seed + 100 + i, rows=rows, cols=cols,
                         kind="normal" if i % 2 == 0 else "beta", n_cand=1600))
    return runs


def planted_specs_for(seed, rows, cols, n=5):
    """Planted biclusters for the batched/served datasets: 1-10% of the rows, 5-16 columns."""
    rng = np.random.default_rng(seed + 7)
    return [(int(rng.integers(max(1, rows // 100), max(2, rows // 10))),
             int(rng.integers(5, min(16, cols) + 1)), bool(i % 3 == 2)) for i in range(n)]


def dataset_from_spec(spec, nan_frac=0.005):
    return make_dataset(spec["seed"], spec["rows"], spec["cols"], kind=spec["kind"],
                        planted=planted_specs_for(spec["seed"], spec["rows"], spec["cols"]),
                        nan_frac=nan_frac, exclude_missing=True, negative=False)

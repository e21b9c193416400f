"""Seeded synthetic rating matrices and initial factors.

This module only draws inputs; it holds none of the ALS arithmetic. Both the
CUDA path and the FP64 oracle take what it returns, so the two always start
from identical data.

Workloads (shapes follow the rating matrices of Sec. 5 and Sec. 6.1, where R
is n_u x n_m with missing entries and integer 1-5 ratings for the
recommender data):

* ``uniform_lowrank``: R = U V^T + N(0, sigma^2) on a uniformly drawn
  fraction of the cells (the small 1000 x 500, n_f = 10 case).
* ``zipf_ratings``: cells drawn from a product of two Zipf(s) popularity laws
  over randomly permuted user and item ranks, deduplicated until exactly
  ``nnz`` distinct cells exist; ratings are clip(rint(3 + u.v + eps), 1, 5)
  with a rank-n_f truth (the 100k x 20k, 10M-entry, n_f = 32 case and its
  larger relatives).

Factor entries of the truth are N(0, 1/sqrt(n_f)) read as a *variance*, so
u.v has unit variance. Observed cells are split 90/10 into train/test.

The initial factor M^(0) ("initialize M randomly", Sec. 2.1 Step 1 and
Algorithm 2) is drawn from a counter-based generator: SplitMix64 (Steele,
Lea and Flood, OOPSLA 2014) feeding the Box-Muller transform, so any element
can be recomputed from (seed, index) alone.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 output for each counter value (uint64 array in, uint64 out).

    State for counter c is seed + (c + 1) * golden; the output is the standard
    SplitMix64 finaliser of that state.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _uniform_open(counter: np.ndarray, seed: int) -> np.ndarray:
    """Uniform doubles in (0, 1]: top 53 bits of SplitMix64, shifted by one ulp."""
    z = splitmix64(counter, seed) >> np.uint64(11)
    return (z.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def init_factor(n: int, f: int, seed: int) -> np.ndarray:
    """Initial factor (n x f, float32) with i.i.d. N(0, 1/sqrt(f)) entries.

    Element e (row-major) uses counters 2e and 2e+1 for the Box-Muller pair and
    keeps the cosine branch.
    """
    e = np.arange(n * f, dtype=np.uint64)
    u1 = _uniform_open(2 * e, seed)
    u2 = _uniform_open(2 * e + np.uint64(1), seed)
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    std = (1.0 / np.sqrt(f)) ** 0.5
    return (z * std).astype(np.float32).reshape(n, f)


@dataclass
class CSR:
    """Compressed rows: int64 indptr, int32 sorted unique indices, float32 values."""
    n_rows: int
    n_cols: int
    indptr: np.ndarray
    indices: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indices.shape[0])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.indptr)


@dataclass
class RatingProblem:
    n_u: int
    n_m: int
    f: int
    train_rows: CSR      # users x items (CSR of train)
    train_cols: CSR      # items x users (CSR of the transpose = CSC of train)
    test_u: np.ndarray   # int32 test user ids
    test_m: np.ndarray   # int32 test item ids
    test_r: np.ndarray   # float32 test ratings
    U_true: np.ndarray
    M_true: np.ndarray


def coo_to_csr(rows: np.ndarray, cols: np.ndarray, vals: np.ndarray,
               n_rows: int, n_cols: int) -> CSR:
    """Build a CSR with indices sorted ascending inside each row."""
    key = rows.astype(np.int64) * np.int64(n_cols) + cols.astype(np.int64)
    order = np.argsort(key, kind="stable")
    r = rows[order]
    counts = np.bincount(r, minlength=n_rows).astype(np.int64)
    indptr = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return CSR(n_rows, n_cols, indptr,
               np.ascontiguousarray(cols[order].astype(np.int32)),
               np.ascontiguousarray(vals[order].astype(np.float32)))


def _truth(n_u: int, n_m: int, f: int, rng: np.random.Generator):
    std = (1.0 / np.sqrt(f)) ** 0.5
    U = rng.standard_normal((n_u, f)) * std
    M = rng.standard_normal((n_m, f)) * std
    return U, M


def _dots(U: np.ndarray, M: np.ndarray, ii: np.ndarray, jj: np.ndarray) -> np.ndarray:
    out = np.empty(ii.shape[0], dtype=np.float64)
    step = 1 << 21
    for s in range(0, ii.shape[0], step):
        out[s:s + step] = np.einsum("ij,ij->i", U[ii[s:s + step]], M[jj[s:s + step]])
    return out


def _split(ii, jj, rr, n_u, n_m, f, U, M, rng, test_frac=0.1) -> RatingProblem:
    n = ii.shape[0]
    perm = rng.permutation(n)
    n_test = int(round(n * test_frac))
    te, tr = perm[:n_test], perm[n_test:]
    rows = coo_to_csr(ii[tr], jj[tr], rr[tr], n_u, n_m)
    cols = coo_to_csr(jj[tr], ii[tr], rr[tr], n_m, n_u)
    return RatingProblem(n_u, n_m, f, rows, cols,
                         ii[te].astype(np.int32), jj[te].astype(np.int32),
                         rr[te].astype(np.float32), U, M)


def uniform_lowrank(n_u: int, n_m: int, f: int, density: float, noise_sd: float,
                    seed: int) -> RatingProblem:
    """R = U V^T + N(0, noise_sd^2) observed on round(density * n_u * n_m) uniform cells."""
    rng = np.random.default_rng(seed)
    U, M = _truth(n_u, n_m, f, rng)
    nnz = int(round(density * n_u * n_m))
    cells = rng.choice(n_u * n_m, size=nnz, replace=False)
    ii = (cells // n_m).astype(np.int64)
    jj = (cells % n_m).astype(np.int64)
    rr = _dots(U, M, ii, jj) + rng.standard_normal(nnz) * noise_sd
    return _split(ii, jj, rr.astype(np.float32), n_u, n_m, f, U, M, rng)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    a = np.sort(a)
    if a.shape[0] == 0:
        return a
    keep = np.empty(a.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def zipf_cells(n_u: int, n_m: int, nnz: int, s_u: float, s_m: float,
               rng: np.random.Generator):
    """Exactly ``nnz`` distinct (user, item) cells from a product of Zipf laws."""
    if nnz > n_u * n_m:
        raise ValueError("more cells requested than the matrix holds")
    pu = 1.0 / np.arange(1, n_u + 1, dtype=np.float64) ** s_u
    pm = 1.0 / np.arange(1, n_m + 1, dtype=np.float64) ** s_m
    pu = pu[rng.permutation(n_u)]
    pm = pm[rng.permutation(n_m)]
    cu = np.cumsum(pu / pu.sum())
    cm = np.cumsum(pm / pm.sum())
    have = np.empty(0, dtype=np.int64)
    while have.shape[0] < nnz:
        want = int((nnz - have.shape[0]) * 2.0) + 1024
        i = np.minimum(np.searchsorted(cu, rng.random(want)), n_u - 1)
        j = np.minimum(np.searchsorted(cm, rng.random(want)), n_m - 1)
        have = _sorted_unique(np.concatenate([have, i.astype(np.int64) * n_m + j]))
    keep = rng.choice(have.shape[0], size=nnz, replace=False)
    cells = have[np.sort(keep)]
    return cells // n_m, cells % n_m


def zipf_ratings(n_u: int, n_m: int, f: int, nnz: int, zipf_s: float,
                 noise_sd: float, seed: int) -> RatingProblem:
    """Integer 1-5 ratings clip(rint(3 + u.v + eps), 1, 5) on Zipf-popular cells."""
    rng = np.random.default_rng(seed)
    U, M = _truth(n_u, n_m, f, rng)
    ii, jj = zipf_cells(n_u, n_m, nnz, zipf_s, zipf_s, rng)
    rr = 3.0 + _dots(U, M, ii, jj) + rng.standard_normal(ii.shape[0]) * noise_sd
    rr = np.clip(np.rint(rr), 1.0, 5.0)
    return _split(ii, jj, rr.astype(np.float32), n_u, n_m, f, U, M, rng)


# Named workloads. "small" is the case the oracle finishes in seconds;
# "zipf_100k" is the 100k x 20k, 10M-entry, n_f = 32 rating matrix.
WORKLOADS = {
    "small": dict(kind="uniform", n_u=1000, n_m=500, f=10, density=0.05,
                  noise_sd=0.1, lam=0.1, budget=0.5, sweeps=10),
    "zipf_100k": dict(kind="zipf", n_u=100_000, n_m=20_000, f=32, nnz=10_000_000,
                      zipf_s=1.0, noise_sd=0.5, lam=0.05, budget=0.25, sweeps=15),
    # 1M x 100k, 10^8 cells, Zipf(0.8), rank-32 truth; drawn on the device
    # (zipf_ratings_device), fitted at n_f = 64 or 128.
    "zipf_1m": dict(kind="zipf_device", n_u=1_000_000, n_m=100_000, f=32, nnz=100_000_000,
                    zipf_s=0.8, noise_sd=0.5, lam=0.05, budget=0.25, sweeps=15),
}


def make_workload(name: str, seed: int = 1, **over) -> RatingProblem:
    w = dict(WORKLOADS[name])
    w.update(over)
    if w["kind"] == "uniform":
        return uniform_lowrank(w["n_u"], w["n_m"], w["f"], w["density"], w["noise_sd"], seed)
    if w["kind"] == "zipf_device":
        raise ValueError(f"{name} is drawn on the device: use zipf_ratings_device")
    return zipf_ratings(w["n_u"], w["n_m"], w["f"], w["nnz"], w["zipf_s"], w["noise_sd"], seed)


# ---------------------------------------------------------------------------
# Device-side generator for the workloads too large to draw on the host in
# reasonable time (10^8 cells). Same recipe as zipf_ratings: Zipf(s) user and
# item popularity with randomly permuted ranks, distinct cells drawn from the
# product law, integer 1-5 ratings clip(rint(3 + u.v + eps), 1, 5) from a
# rank-`f` truth with N(0, 1/sqrt(f)) (variance) entries, 90/10 train/test.
# Seeded through torch's counter-based CUDA generator, so a (seed, sizes,
# torch build) triple gives the same matrix; it is not the host generator's
# stream, so its matrices differ from zipf_ratings' for the same seed.
@dataclass
class DeviceRatingProblem:
    n_u: int
    n_m: int
    f: int
    rows: tuple   # (indptr int64, indices int32, values float32) of train, users x items
    cols: tuple   # the same for items x users
    test_u: "object"
    test_m: "object"
    test_r: "object"


def zipf_ratings_device(n_u: int, n_m: int, f: int, nnz: int, zipf_s: float, noise_sd: float, seed: int,
                        device="cuda") -> DeviceRatingProblem:
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    std = (1.0 / np.sqrt(f)) ** 0.5
    U = torch.randn((n_u, f), generator=g, device=device) * std
    M = torch.randn((n_m, f), generator=g, device=device) * std

    def cdf(n):
        w = 1.0 / torch.arange(1, n + 1, dtype=torch.float64, device=device) ** zipf_s
        w = w[torch.randperm(n, generator=g, device=device)]
        return torch.cumsum(w / w.sum(), 0)

    cu, cm = cdf(n_u), cdf(n_m)
    if nnz > n_u * n_m:
        raise ValueError("more cells requested than the matrix holds")
    have = torch.empty(0, dtype=torch.int64, device=device)
    for _ in range(1000):
        if have.numel() >= nnz:
            break
        want = int((nnz - have.numel()) * 1.3) + 1024
        i = torch.clamp(torch.searchsorted(cu, torch.rand(want, generator=g, device=device, dtype=torch.float64)),
                        max=n_u - 1)
        j = torch.clamp(torch.searchsorted(cm, torch.rand(want, generator=g, device=device, dtype=torch.float64)),
                        max=n_m - 1)
        have = torch.unique(torch.cat([have, i * n_m + j]))
    if have.numel() < nnz:
        raise ValueError("the popularity law leaves too few distinct cells for nnz")
    keep = torch.randperm(have.numel(), generator=g, device=device)[:nnz]
    cells = have[torch.sort(keep).values]
    del have, keep
    ii, jj = cells // n_m, cells % n_m
    rr = torch.empty(nnz, dtype=torch.float32, device=device)
    step = 1 << 23
    for s in range(0, nnz, step):
        a, b = ii[s:s + step], jj[s:s + step]
        rr[s:s + step] = (U[a] * M[b]).sum(1)
    rr = torch.clamp(torch.round(3.0 + rr + torch.randn(nnz, generator=g, device=device) * noise_sd), 1.0, 5.0)
    is_test = torch.zeros(nnz, dtype=torch.bool, device=device)
    is_test[torch.randperm(nnz, generator=g, device=device)[:int(round(nnz * 0.1))]] = True
    tr = ~is_test

    def csr(r_idx, c_idx, vals, n_rows, n_cols):
        key = r_idx * n_cols + c_idx
        order = torch.argsort(key)
        counts = torch.bincount(r_idx, minlength=n_rows)
        indptr = torch.zeros(n_rows + 1, dtype=torch.int64, device=device)
        indptr[1:] = torch.cumsum(counts, 0)
        return indptr, c_idx[order].to(torch.int32).contiguous(), vals[order].contiguous()

    rows = csr(ii[tr], jj[tr], rr[tr], n_u, n_m)
    cols = csr(jj[tr], ii[tr], rr[tr], n_m, n_u)
    return DeviceRatingProblem(n_u, n_m, f, rows, cols, ii[is_test].to(torch.int32), jj[is_test].to(torch.int32),
                               rr[is_test])


# ---------------------------------------------------------------------------
# Small single-side cases for kernel captures: rows of one length band with
# distinct sorted column ids, N(0, 1) ratings and Y ~ N(0, 0.6^2) (30,000
# columns). They isolate one row bucket of the half-sweep.
CAPTURE_CASES = {
    "rows1_32": (60_000, 1, 32),
    "rows33_128": (20_000, 33, 128),
    "rows129_512": (6_000, 129, 512),
    "rows513_1024": (3_000, 513, 1024),
    "split": (300, 2_000, 20_000),
}


def capture_case(name: str, f: int, seed: int = 0, n_cols: int = 30_000):
    n_rows, lo, hi = CAPTURE_CASES[name]
    rng = np.random.default_rng(seed)
    lengths = rng.integers(lo, hi + 1, n_rows)
    indptr = np.zeros(n_rows + 1, np.int64)
    np.cumsum(lengths, out=indptr[1:])
    idx = np.concatenate([np.sort(rng.choice(n_cols, size=int(L), replace=False)) for L in lengths])
    vals = rng.standard_normal(int(lengths.sum())).astype(np.float32)
    Y = (rng.standard_normal((n_cols, f)) * 0.6).astype(np.float32)
    return CSR(n_rows, n_cols, indptr, idx.astype(np.int32), vals), Y


# ---------------------------------------------------------------------------
# The simulation design of Sec. 5.1: factors U (n_u x p) and M (n_m x p) with
# i.i.d. rows from D1 N(0, Sigma), D2 the log-normal exp(N(0, Sigma)) or D3
# the multivariate t with 4 degrees of freedom N(0, Sigma) / sqrt(chi2_4 / 4),
# Sigma_ij = 0.6^|i - j|; R^o = U M^T; R = R^o + N(0, 1) noise on every cell;
# then a fraction `missing` of the cells is removed at random. The removed
# cells form the prediction set I^c (their values are those of R), the rest
# the empirical set I used for fitting.
#
# Reading of a garbled point: the paper removes "(1 - alpha)" of the cells
# yet calls alpha = 0.4 (R1) the dense case and alpha = 0.7 (R4) the sparse
# one; `missing` = alpha is the fraction removed, which matches R1 dense,
# R4 sparse.
SIM_DISTRIBUTIONS = ("D1", "D2", "D3")
SIM_MISSING = {"R1": 0.4, "R2": 0.5, "R3": 0.6, "R4": 0.7}


@dataclass
class SimulationProblem:
    n_u: int
    n_m: int
    f: int
    train_rows: CSR      # empirical set I, users x items
    train_cols: CSR      # its transpose
    pred_u: np.ndarray   # prediction set I^c: int32 users
    pred_m: np.ndarray   # int32 items
    pred_r: np.ndarray   # float32 values of R there
    U_true: np.ndarray
    M_true: np.ndarray


def _sim_factor(n: int, p: int, dist: str, rng: np.random.Generator) -> np.ndarray:
    idx = np.arange(p)
    sigma = 0.6 ** np.abs(idx[:, None] - idx[None, :])
    L = np.linalg.cholesky(sigma)
    z = rng.standard_normal((n, p)) @ L.T
    if dist == "D1":
        return z
    if dist == "D2":
        return np.exp(z)
    if dist == "D3":
        w = rng.chisquare(4.0, size=(n, 1))
        return z / np.sqrt(w / 4.0)
    raise ValueError(f"unknown factor distribution {dist!r}")


def simulation(dist: str = "D1", missing: float = 0.4, n_u: int = 3600, n_m: int = 3600, f: int = 60,
               seed: int = 1) -> SimulationProblem:
    rng = np.random.default_rng(seed)
    U = _sim_factor(n_u, f, dist, rng)
    M = _sim_factor(n_m, f, dist, rng)
    R = U @ M.T + rng.standard_normal((n_u, n_m))
    n_cells = n_u * n_m
    n_miss = int(round(missing * n_cells))
    gone = np.zeros(n_cells, bool)
    gone[rng.choice(n_cells, size=n_miss, replace=False)] = True
    cells = np.arange(n_cells, dtype=np.int64)
    obs, mis = cells[~gone], cells[gone]
    flat = R.reshape(-1)
    ii, jj = obs // n_m, obs % n_m
    rows = coo_to_csr(ii, jj, flat[obs].astype(np.float32), n_u, n_m)
    cols = coo_to_csr(jj, ii, flat[obs].astype(np.float32), n_m, n_u)
    return SimulationProblem(n_u, n_m, f, rows, cols, (mis // n_m).astype(np.int32), (mis % n_m).astype(np.int32),
                             flat[mis].astype(np.float32), U, M)


def relevant_items(n_u: int, n_m: int, test_u: np.ndarray, test_m: np.ndarray, test_r: np.ndarray,
                   threshold: float) -> CSR:
    """Per user, the held-out items whose true rating is at least `threshold`
    (the items that should be recommended), as a CSR of sorted item ids."""
    keep = np.asarray(test_r) >= threshold
    u = np.asarray(test_u)[keep].astype(np.int64)
    m = np.asarray(test_m)[keep].astype(np.int64)
    return coo_to_csr(u, m, np.ones(u.shape[0], np.float32), n_u, n_m)


def top_share_threshold(values: np.ndarray, share: float = 0.05) -> float:
    """The value above which the largest `share` of `values` lie (the
    relevance cut of the simulation's recommendation metrics)."""
    v = np.sort(np.asarray(values, np.float64))
    return float(v[int(np.floor((1.0 - share) * (v.shape[0] - 1)))]) if v.size else np.inf

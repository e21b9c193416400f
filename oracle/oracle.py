"""ctypes front end of the FP64 C oracle (``core_als_oracle.c``) plus the
Algorithm 2 sweep loop.

TEST INFRASTRUCTURE ONLY. Nothing in the CUDA product path imports this.

Functions and what pins each one (tests/test_oracle_pins.py):

* ``budget``            s = floor(n r), or min(n, s_fixed) (fixed subsample
                        size): pinned by hand values incl. r = 0.29.
* ``ces_row``           Algorithm 1: pinned by brute force over all subsets on
                        tiny rows and by hand-worked golden rows.
* ``half_sweep``        Eq. (core_ui)/(core_mj), Eq. (U format)/(M format):
                        full and symmetric modes pinned to Householder-QR
                        ridge least squares; asymmetric mode pinned by the
                        hand-worked f = 1 and f = 2 golden examples, and by the
                        row-subset reduction (when every column keeps the same
                        rows, X*^T X = X_K^T X_K, a QR-solvable ridge problem).
* ``fit``               Algorithm 2: full ALS pinned by a non-increasing
                        objective (Sec. 2.1) and exact recovery of a noiseless,
                        fully observed rank-n_f matrix; r = 1 reduces to full.
* ``factor_sketch`` / ``sketch="factor"``: the fast variant (CES once on the
                        whole design factor): pinned by its reduction to the
                        per-slice estimator on fully observed matrices, by the
                        row-subset reduction to QR ridge, and r = 1 = full.
* ``objective``, ``rmse``: pinned by a hand-computed example.
* ``remse``             Sec. 5.1 relative error: hand example, exact fit = 0,
                        zero prediction = 1.
* ``rank_topk`` / ``rank_metrics``: Hit@k, NDCG@k of Sec. 5.1: hand-worked
                        golden case, brute-force ranking of exactly
                        representable scores, closed forms (all relevant).
* ``solve_batch``       LU / Cholesky: pinned against LAPACK (numpy) and
                        Cramer's rule at f = 2.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "core_als_oracle.c"
_LIB = _HERE / "_build" / "libcore_als_oracle.so"

REG_WEIGHTED, REG_PLAIN = 0, 1
GRAM_ASYM, GRAM_SYM, GRAM_FULL = 0, 1, 2
FLAG_RATIO, FLAG_SINGULAR = 1, 2


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP when available)."""
    _LIB.parent.mkdir(parents=True, exist_ok=True)
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", str(_SRC), "-o", str(_LIB) + ".tmp", "-lm"]
    r = subprocess.run(base[:4] + ["-fopenmp"] + base[4:] + ["-fopenmp"], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(str(_LIB) + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(str(path))
        P = C.c_void_p
        i64, f64, i32 = C.c_int64, C.c_double, C.c_int
        L.oracle_budget.restype = i64
        L.oracle_budget.argtypes = [i64, f64, i64, i64]
        L.oracle_ces.restype = None
        L.oracle_ces.argtypes = [i64, i32, P, i64, P, P]
        L.oracle_assemble.restype = None
        L.oracle_assemble.argtypes = [i64, i32, P, P, P, i32, f64, P, P]
        L.oracle_solve_lu.restype = i32
        L.oracle_solve_lu.argtypes = [i32, P, P, P, f64, P]
        L.oracle_solve_chol.restype = i32
        L.oracle_solve_chol.argtypes = [i32, P, P, P, f64, P]
        L.oracle_half_sweep.restype = i32
        L.oracle_half_sweep.argtypes = [i64, P, P, P, P, i32, P, f64, f64, i64, i64, i32, i32, f64, P, P, P, P]
        L.oracle_select_half.restype = i32
        L.oracle_select_half.argtypes = [i64, P, P, i32, P, f64, i64, i64, P, P]
        L.oracle_assemble_half.restype = i32
        L.oracle_assemble_half.argtypes = [i64, P, P, P, i32, P, f64, f64, i64, i64, i32, i32, P, P, P]
        L.oracle_factor_sketch.restype = i32
        L.oracle_factor_sketch.argtypes = [i64, i32, P, f64, i64, i64, P]
        L.oracle_remse.restype = f64
        L.oracle_remse.argtypes = [i64, P, P, P, i32, P, P]
        L.oracle_rank_topk.restype = i32
        L.oracle_rank_topk.argtypes = [i64, i64, i32, P, P, P, P, i32, P]
        L.oracle_rank_metrics.restype = None
        L.oracle_rank_metrics.argtypes = [i64, P, i32, i32, i32, P, P, P, P, P]
        L.oracle_solve_batch.restype = None
        L.oracle_solve_batch.argtypes = [i64, i32, P, P, i32, f64, P, P, P]
        L.oracle_sse.restype = f64
        L.oracle_sse.argtypes = [i64, P, P, P, i32, P, P]
        L.oracle_reg_term.restype = f64
        L.oracle_reg_term.argtypes = [i64, P, i32, P, f64, i32]
        L.oracle_num_threads.restype = i32
        L.oracle_set_threads.restype = None
        L.oracle_set_threads.argtypes = [i32]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def budget(n: int, r: float, min_keep: int = 0, fixed_keep: int = 0) -> int:
    """s = floor(n * r) (Sec. 3 selection rule), or min(n, fixed_keep) when
    fixed_keep > 0 (fixed subsample size); optionally raised to min_keep."""
    return int(lib().oracle_budget(int(n), float(r), int(min_keep), int(fixed_keep)))


def factor_sketch(Y, r: float, min_keep: int = 0, fixed_keep: int = 0) -> np.ndarray:
    """Fast variant (Sec. 3): CES on the whole design factor Y (n_other x f)
    with s = budget(n_other); returns the 0/1 keep matrix (uint8)."""
    Y = _c(Y, np.float64)
    n, f = Y.shape
    keep = np.zeros((n, f), np.uint8)
    if lib().oracle_factor_sketch(n, f, _p(Y), float(r), int(min_keep), int(fixed_keep), _p(keep)) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return keep


def _keep_arg(sketch, Y, r, min_keep, fixed_keep):
    """(holder, pointer) of the factor-wide keep matrix of the fast variant,
    or (None, None) for the per-slice CES of Algorithm 2."""
    if sketch == "slice":
        return None, None
    if sketch != "factor":
        raise ValueError("sketch must be 'slice' or 'factor'")
    k = factor_sketch(Y, r, min_keep, fixed_keep)
    return k, _p(k)


def ces_row(X: np.ndarray, s: int) -> np.ndarray:
    """Algorithm 1 on one slice X (n x f); returns the 0/1 keep matrix (uint8)."""
    X = _c(X, np.float64)
    n, f = X.shape
    keep = np.zeros((n, f), dtype=np.uint8)
    scratch = np.zeros(max(n, 1) * 16, dtype=np.uint8)
    lib().oracle_ces(n, f, _p(X), int(s), _p(keep), _p(scratch))
    return keep


def assemble_row(X, r, keep, gram_mode: int, reg: float):
    """Normal equations of one row: (G, b) with reg added on the diagonal."""
    X = _c(X, np.float64)
    n, f = X.shape
    r = _c(r, np.float64)
    keep = _c(keep, np.uint8) if keep is not None else np.ones((n, f), np.uint8)
    G = np.zeros((f, f))
    b = np.zeros(f)
    lib().oracle_assemble(n, f, _p(X), _p(r), _p(keep), int(gram_mode), float(reg), _p(G), _p(b))
    return G, b


def solve_batch(G: np.ndarray, b: np.ndarray, method: int = 0, ratio_max: float = 1e6):
    """Batched LU (method 0) or Cholesky (method 1); returns (X, flags, ratios)."""
    G = _c(G, np.float64)
    b = _c(b, np.float64)
    n, f = b.shape
    X = np.zeros((n, f))
    flags = np.zeros(n, np.int32)
    ratios = np.zeros(n)
    lib().oracle_solve_batch(n, f, _p(G), _p(b), int(method), float(ratio_max), _p(X), _p(flags), _p(ratios))
    return X, flags, ratios


def half_sweep(indptr, indices, values, Y, lam: float, r: float, gram_mode: int = GRAM_ASYM,
               reg_mode: int = REG_WEIGHTED, min_keep: int = 0, ratio_max: float = 1e6,
               rows=None, fixed_keep: int = 0, sketch: str = "slice"):
    """One half-sweep (Algorithm 2 inner loop for one side). Returns (X, flags, ratios).

    ``rows`` restricts the update to a subset of rows (others are left zero).
    ``sketch="factor"`` is the fast variant (CES once on the whole Y).
    """
    indptr = _c(indptr, np.int64)
    indices = _c(indices, np.int32)
    values = _c(values, np.float32)
    Y = _c(Y, np.float64)
    n_rows = indptr.shape[0] - 1
    f = Y.shape[1]
    X = np.zeros((n_rows, f))
    flags = np.zeros(n_rows, np.int32)
    ratios = np.zeros(n_rows)
    if rows is None:
        cnt, rp = n_rows, None
    else:
        rows = _c(rows, np.int64)
        cnt, rp = rows.shape[0], _p(rows)
    hold, kp = _keep_arg(sketch, Y, r, min_keep, fixed_keep)
    rc = lib().oracle_half_sweep(cnt, rp, _p(indptr), _p(indices), _p(values), f, _p(Y), float(lam),
                                 float(r), int(min_keep), int(fixed_keep), int(reg_mode), int(gram_mode),
                                 float(ratio_max), kp, _p(X), _p(flags), _p(ratios))
    del hold
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return X, flags, ratios


def select_half(indptr, indices, Y, r: float, min_keep: int = 0, fixed_keep: int = 0,
                sketch: str = "slice") -> np.ndarray:
    """Packed CES masks, uint32[nnz, ceil(f/32)] (bit a%32 of word a//32)."""
    indptr = _c(indptr, np.int64)
    indices = _c(indices, np.int32)
    Y = _c(Y, np.float64)
    f = Y.shape[1]
    words = (f + 31) // 32
    masks = np.zeros((indices.shape[0], words), np.uint32)
    hold, kp = _keep_arg(sketch, Y, r, min_keep, fixed_keep)
    rc = lib().oracle_select_half(indptr.shape[0] - 1, _p(indptr), _p(indices), f, _p(Y), float(r),
                                  int(min_keep), int(fixed_keep), kp, _p(masks))
    del hold
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return masks


def assemble_half(indptr, indices, values, Y, lam: float, r: float, gram_mode: int = GRAM_ASYM,
                  reg_mode: int = REG_WEIGHTED, min_keep: int = 0, fixed_keep: int = 0, sketch: str = "slice"):
    """(G, b) of every row: G is n_rows x f x f, b is n_rows x f."""
    indptr = _c(indptr, np.int64)
    indices = _c(indices, np.int32)
    values = _c(values, np.float32)
    Y = _c(Y, np.float64)
    n_rows = indptr.shape[0] - 1
    f = Y.shape[1]
    G = np.zeros((n_rows, f, f))
    b = np.zeros((n_rows, f))
    hold, kp = _keep_arg(sketch, Y, r, min_keep, fixed_keep)
    rc = lib().oracle_assemble_half(n_rows, _p(indptr), _p(indices), _p(values), f, _p(Y), float(lam),
                                    float(r), int(min_keep), int(fixed_keep), int(reg_mode), int(gram_mode), kp,
                                    _p(G), _p(b))
    del hold
    if rc != 0:
        raise MemoryError("oracle scratch allocation failed")
    return G, b


def sse(iu, im, r, U, M) -> float:
    """Sum over entries of (r - u_i . m_j)^2."""
    iu = _c(iu, np.int32)
    im = _c(im, np.int32)
    r = _c(r, np.float32)
    U = _c(U, np.float64)
    M = _c(M, np.float64)
    return float(lib().oracle_sse(iu.shape[0], _p(iu), _p(im), _p(r), U.shape[1], _p(U), _p(M)))


def rmse(iu, im, r, U, M) -> float:
    n = len(r)
    return float(np.sqrt(sse(iu, im, r, U, M) / n)) if n else 0.0


def csr_to_coo(indptr, indices):
    rows = np.repeat(np.arange(len(indptr) - 1, dtype=np.int32), np.diff(indptr))
    return rows, np.asarray(indices, dtype=np.int32)


def objective(rows_csr, cols_csr, U, M, lam: float, reg_mode: int = REG_WEIGHTED) -> float:
    """Eq. (object function): data term over the training entries plus the
    weighted-lambda terms lambda (sum_i n_ui |u_i|^2 + sum_j n_mj |m_j|^2);
    with the plain regulariser lambda (sum_i |u_i|^2 + sum_j |m_j|^2)."""
    iu, im = csr_to_coo(rows_csr.indptr, rows_csr.indices)
    data = sse(iu, im, rows_csr.values, U, M)
    L = lib()
    Uc = _c(U, np.float64)
    Mc = _c(M, np.float64)
    ru = L.oracle_reg_term(rows_csr.n_rows, _p(_c(rows_csr.indptr, np.int64)), U.shape[1], _p(Uc), float(lam),
                           int(reg_mode))
    rm = L.oracle_reg_term(cols_csr.n_rows, _p(_c(cols_csr.indptr, np.int64)), M.shape[1], _p(Mc), float(lam),
                           int(reg_mode))
    return data + ru + rm


def remse(iu, im, r, U, M) -> float:
    """Sec. 5.1: sqrt(sum_E (r - u_i . m_j)^2) / sqrt(sum_E r^2) over the
    entries E (the empirical set for ReMSE, the prediction set for P-ReMSE)."""
    iu = _c(iu, np.int32)
    im = _c(im, np.int32)
    r = _c(r, np.float32)
    U = _c(U, np.float64)
    M = _c(M, np.float64)
    return float(lib().oracle_remse(iu.shape[0], _p(iu), _p(im), _p(r), U.shape[1], _p(U), _p(M)))


def rank_topk(U, M, train_indptr, train_indices, K: int) -> np.ndarray:
    """Per user the K unrated items of largest FP32 predicted rating (ties:
    lower item first), int32[n_u, K] (-1 pads)."""
    U = _c(U, np.float32)
    M = _c(M, np.float32)
    ip = _c(train_indptr, np.int64)
    ix = _c(train_indices, np.int32)
    n_u, f = U.shape
    out = np.zeros((n_u, int(K)), np.int32)
    if lib().oracle_rank_topk(n_u, M.shape[0], f, _p(U), _p(M), _p(ip), _p(ix), int(K), _p(out)) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return out


def rank_metrics(topk, rel_indptr, rel_indices, k_hit: int = 5, k_ndcg: int = 10):
    """(Hit@k_hit, NDCG@k_ndcg, users evaluated) of the lists topk against
    the relevant items (CSR per user)."""
    topk = _c(topk, np.int32)
    ip = _c(rel_indptr, np.int64)
    ix = _c(rel_indices, np.int32)
    hit, ndcg, n = C.c_double(), C.c_double(), C.c_int64()
    lib().oracle_rank_metrics(topk.shape[0], _p(topk), topk.shape[1], int(k_hit), int(k_ndcg), _p(ip), _p(ix),
                              C.byref(hit), C.byref(ndcg), C.byref(n))
    return hit.value, ndcg.value, n.value


def fit(rows_csr, cols_csr, M0, lam: float, r: float, sweeps: int, gram_mode: int = GRAM_ASYM,
        reg_mode: int = REG_WEIGHTED, min_keep: int = 0, ratio_max: float = 1e6, callback=None,
        fixed_keep: int = 0, sketch: str = "slice"):
    """Algorithm 2 (Core-ALS), or Steps 1-4 of Sec. 2.1 when gram_mode is FULL.

    Starting from M^(0) = M0: every sweep updates all users from the current
    M (Eq. core_ui), then all items from the *new* U (Eq. core_mj).
    callback(t, U, M) is called after each sweep. Returns (U, M).
    """
    M = np.asarray(M0, dtype=np.float64).copy()
    U = np.zeros((rows_csr.n_rows, M.shape[1]))
    for t in range(sweeps):
        U, _, _ = half_sweep(rows_csr.indptr, rows_csr.indices, rows_csr.values, M, lam, r,
                             gram_mode, reg_mode, min_keep, ratio_max, fixed_keep=fixed_keep, sketch=sketch)
        M, _, _ = half_sweep(cols_csr.indptr, cols_csr.indices, cols_csr.values, U, lam, r,
                             gram_mode, reg_mode, min_keep, ratio_max, fixed_keep=fixed_keep, sketch=sketch)
        if callback is not None:
            callback(t, U, M)
    return U, M


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

"""Shared test helpers: seeded hand-shaped problems (no ALS arithmetic here)."""
import numpy as np

from paper_2509_18024_gb300 import synth


def rows_problem(lengths, n_cols, f, seed, pool=None, rating_pool=None):
    """CSR with the given row lengths (distinct sorted column ids per row),
    ratings and an other-side factor Y (n_cols x f, float32). With `pool`,
    Y entries are drawn from that finite set (many ties)."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, np.int64)
    assert lengths.max(initial=0) <= n_cols
    indptr = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=indptr[1:])
    idx = np.concatenate([np.sort(rng.choice(n_cols, size=int(L), replace=False)) for L in lengths]
                         ) if lengths.sum() else np.zeros(0, np.int64)
    if rating_pool is None:
        vals = rng.standard_normal(int(lengths.sum()))
    else:
        vals = rng.choice(rating_pool, size=int(lengths.sum()))
    if pool is None:
        Y = rng.standard_normal((n_cols, f)) * 0.6
    else:
        Y = rng.choice(np.asarray(pool, np.float64), size=(n_cols, f))
    csr = synth.CSR(len(lengths), n_cols, indptr, idx.astype(np.int32), vals.astype(np.float32))
    return csr, Y.astype(np.float32)


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))

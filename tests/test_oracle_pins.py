"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: each compares it with an
independent route (Householder QR from LAPACK, brute force over subsets,
hand-worked golden rows, closed forms, or invariants stated in the paper).
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2509_18024_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "core_rows.json")


def one_row_csr(X, r):
    """A 1-row problem whose design slice is exactly X: Y = X, indices 0..n-1."""
    n = X.shape[0]
    return (np.array([0, n], np.int64), np.arange(n, dtype=np.int32),
            np.asarray(r, np.float32), np.asarray(X, np.float64))


def ridge_qr(X, r, reg):
    """Ridge regression by Householder QR of [X; sqrt(reg) I] against [r; 0]."""
    n, f = X.shape
    A = np.vstack([X, np.sqrt(reg) * np.eye(f)])
    y = np.concatenate([r, np.zeros(f)])
    Q, R = np.linalg.qr(A)
    return np.linalg.solve(R, Q.T @ y)


# --------------------------------------------------------------------- budget
def test_budget_floor(oracle_mod):
    # Sec. 3: floor(|I_i| * r). 100 * 0.29 is 28.999999999999996 in IEEE double.
    assert oracle_mod.budget(100, 0.29) == 28
    assert oracle_mod.budget(4, 0.5) == 2
    assert oracle_mod.budget(3, 0.5) == 1
    assert oracle_mod.budget(3, 0.25) == 0
    assert oracle_mod.budget(7, 0.25) == 1
    assert oracle_mod.budget(10, 1.0) == 10
    assert oracle_mod.budget(0, 0.5) == 0
    assert oracle_mod.budget(3, 0.25, min_keep=2) == 2
    assert oracle_mod.budget(1, 0.25, min_keep=2) == 1


# ------------------------------------------------------------------ selection
def brute_force_keep(col, s):
    """The unique size-s subset K with min_K |x| >= max_not-K |x| and, among
    equal |x| across the boundary, kept positions below dropped ones."""
    n = len(col)
    mags = np.abs(col)
    found = []
    for K in itertools.combinations(range(n), s):
        Ks = set(K)
        ok = True
        for k in Ks:
            for j in range(n):
                if j in Ks:
                    continue
                if mags[k] < mags[j] or (mags[k] == mags[j] and k > j):
                    ok = False
        if ok:
            found.append(Ks)
    assert len(found) == 1
    out = np.zeros(n, np.uint8)
    out[list(found[0])] = 1
    return out


@pytest.mark.parametrize("seed", range(12))
def test_ces_matches_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    f = int(rng.integers(1, 5))
    pool = np.array([-2.0, -1.0, -0.0, 0.0, 1.0, 2.0, 0.5, -0.5])
    X = rng.choice(pool, size=(n, f))
    for s in range(n + 1):
        keep = oracle_mod.ces_row(X, s)
        for a in range(f):
            assert np.array_equal(keep[:, a], brute_force_keep(X[:, a], s)), (seed, s, a)


def test_ces_golden(oracle_mod):
    g = json.load(open(GOLDEN))
    for c in g["cases"]:
        X = np.array(c["X"])
        s = oracle_mod.budget(X.shape[0], c["budget"])
        assert np.array_equal(oracle_mod.ces_row(X, s), np.array(c["keep"], np.uint8)), c["name"]


# ------------------------------------------------------------- the estimator
@pytest.mark.parametrize("case", ["f1_basic", "f1_ties", "f2_asym"])
def test_golden_rows(oracle_mod, case):
    g = {c["name"]: c for c in json.load(open(GOLDEN))["cases"]}[case]
    X = np.array(g["X"])
    indptr, idx, vals, Y = one_row_csr(X, g["r"])
    for mode, key in ((oracle_mod.GRAM_ASYM, "x_asym"), (oracle_mod.GRAM_SYM, "x_sym"),
                      (oracle_mod.GRAM_FULL, "x_full")):
        if key not in g:
            continue
        x, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, g["lam"], g["budget"], mode)
        np.testing.assert_allclose(x[0], g[key], rtol=1e-14, atol=0, err_msg=f"{case} {key}")


@pytest.mark.parametrize("seed", range(6))
def test_full_update_is_ridge_qr(oracle_mod, seed):
    """Eq. (U format) is ridge regression with penalty lambda n_i: it equals
    least squares on the augmented system, solved here by Householder QR."""
    rng = np.random.default_rng(100 + seed)
    n, f = int(rng.integers(3, 40)), int(rng.integers(1, 9))
    X = rng.standard_normal((n, f))
    r = rng.standard_normal(n).astype(np.float32)
    lam = float(rng.uniform(0.01, 0.5))
    indptr, idx, vals, Y = one_row_csr(X, r)
    x, flags, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, 1.0, oracle_mod.GRAM_FULL)
    ref = ridge_qr(X, r.astype(np.float64), lam * n)
    np.testing.assert_allclose(x[0], ref, rtol=1e-11, atol=1e-13)
    # PLAIN regulariser: lambda alone.
    x2, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, 1.0, oracle_mod.GRAM_FULL,
                                     reg_mode=oracle_mod.REG_PLAIN)
    np.testing.assert_allclose(x2[0], ridge_qr(X, r.astype(np.float64), lam), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_sym_update_is_ridge_on_sketch(oracle_mod, seed):
    """The symmetric variant (X*^T X* + lambda n E) x = X*^T r is ridge
    regression with the sketch X* as design: QR on [X*; sqrt(lambda n) I]."""
    rng = np.random.default_rng(200 + seed)
    n, f = int(rng.integers(4, 30)), int(rng.integers(1, 6))
    X = rng.standard_normal((n, f))
    r = rng.standard_normal(n).astype(np.float32)
    lam, budget = 0.2, float(rng.uniform(0.3, 0.9))
    s = oracle_mod.budget(n, budget)
    keep = np.stack([brute_force_keep(X[:, a], s) for a in range(f)], axis=1)
    indptr, idx, vals, Y = one_row_csr(X, r)
    x, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, budget, oracle_mod.GRAM_SYM)
    ref = ridge_qr(X * keep, r.astype(np.float64), lam * n)
    np.testing.assert_allclose(x[0], ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_asym_row_subset_reduction(oracle_mod, seed):
    """When every column keeps the same rows K, X* = D_K X and the paper's
    asymmetric X*^T X equals X_K^T X_K: the update is ridge on the rows in K
    with the penalty still lambda * (full n)."""
    rng = np.random.default_rng(300 + seed)
    n, f = int(rng.integers(6, 30)), int(rng.integers(1, 6))
    budget = float(rng.uniform(0.2, 0.8))
    s = int(np.floor(n * budget))
    K = rng.choice(n, size=s, replace=False)
    X = rng.uniform(-1, 1, (n, f))
    X[K] = rng.uniform(2, 3, (s, f)) * rng.choice([-1.0, 1.0], (s, f))
    r = rng.standard_normal(n).astype(np.float32)
    lam = 0.3
    indptr, idx, vals, Y = one_row_csr(X, r)
    x, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, budget, oracle_mod.GRAM_ASYM)
    ref = ridge_qr(X[K], r.astype(np.float64)[K], lam * n) if s else np.zeros(f)
    np.testing.assert_allclose(x[0], ref, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("seed", range(8))
def test_nf1_closed_form(oracle_mod, seed):
    """n_f = 1: x = sum_S x_k r_k / (sum_S x_k^2 + lambda n), S = top-s by |x|."""
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(1, 25))
    col = rng.standard_normal(n)
    r = rng.standard_normal(n).astype(np.float32)
    lam, budget = 0.15, float(rng.uniform(0.05, 1.0))
    s = oracle_mod.budget(n, budget)
    order = sorted(range(n), key=lambda k: (-abs(col[k]), k))[:s]
    num = sum(col[k] * float(r[k]) for k in order)
    den = sum(col[k] ** 2 for k in order) + lam * n
    indptr, idx, vals, Y = one_row_csr(col[:, None], r)
    x, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, budget, oracle_mod.GRAM_ASYM)
    assert x[0, 0] == pytest.approx(num / den, rel=1e-13, abs=1e-300)


def test_budget_all_equals_full(oracle_mod):
    """r = 1 gives S = all ones, so Eq. (core_ui) collapses to Eq. (U format)."""
    p = synth.make_workload("small")
    M0 = synth.init_factor(p.n_m, p.f, 7)
    R = p.train_rows
    xa, _, _ = oracle_mod.half_sweep(R.indptr, R.indices, R.values, M0, 0.1, 1.0, oracle_mod.GRAM_ASYM)
    xs, _, _ = oracle_mod.half_sweep(R.indptr, R.indices, R.values, M0, 0.1, 1.0, oracle_mod.GRAM_SYM)
    xf, _, _ = oracle_mod.half_sweep(R.indptr, R.indices, R.values, M0, 0.1, 1.0, oracle_mod.GRAM_FULL)
    np.testing.assert_allclose(xa, xf, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(xs, xf, rtol=1e-10, atol=1e-12)


def test_zero_budget_gives_zero(oracle_mod):
    """s = 0 keeps nothing: G = lambda n E, b = 0, so x = 0."""
    X = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, -6.0]])
    indptr, idx, vals, Y = one_row_csr(X, [1.0, 2.0, 3.0])
    x, flags, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, 0.1, 0.3, oracle_mod.GRAM_ASYM)
    assert np.all(x == 0) and flags[0] == 0


# -------------------------------------------------------------------- solves
@pytest.mark.parametrize("seed", range(4))
def test_lu_and_cholesky_against_lapack(oracle_mod, seed):
    rng = np.random.default_rng(500 + seed)
    f, m = 12, 20
    A = rng.standard_normal((m, f, f)) + 4 * np.eye(f)
    b = rng.standard_normal((m, f))
    x, flags, _ = oracle_mod.solve_batch(A, b, method=0)
    np.testing.assert_allclose(x, np.linalg.solve(A, b[..., None])[..., 0], rtol=1e-11, atol=1e-12)
    S = A @ np.transpose(A, (0, 2, 1)) + np.eye(f)
    x, flags, _ = oracle_mod.solve_batch(S, b, method=1)
    np.testing.assert_allclose(x, np.linalg.solve(S, b[..., None])[..., 0], rtol=1e-11, atol=1e-12)
    assert np.all(flags == 0)


def test_lu_cramer_2x2_needs_pivot(oracle_mod):
    # Zero leading pivot: only correct with row exchange.
    G = np.array([[[0.0, 2.0], [3.0, 1.0]]])
    b = np.array([[4.0, 5.0]])
    x, flags, ratios = oracle_mod.solve_batch(G, b, method=0)
    det = 0.0 * 1.0 - 2.0 * 3.0
    np.testing.assert_allclose(x[0], [(4 * 1 - 2 * 5) / det, (0 * 5 - 3 * 4) / det], rtol=1e-15)
    assert ratios[0] == pytest.approx(3.0 / 2.0)


def test_singular_and_ratio_flags(oracle_mod):
    G = np.array([np.zeros((2, 2)), np.diag([1.0, 1e-7]), np.diag([1.0, 1e-5])])
    b = np.ones((3, 2))
    x, flags, ratios = oracle_mod.solve_batch(G, b, method=0, ratio_max=1e6)
    assert flags[0] & oracle_mod.FLAG_SINGULAR and np.all(x[0] == 0)
    assert flags[1] == oracle_mod.FLAG_RATIO and ratios[1] == pytest.approx(1e7)
    assert flags[2] == 0
    x, flags, ratios = oracle_mod.solve_batch(G[1:], b[1:], method=1, ratio_max=1e6)
    assert flags[0] == oracle_mod.FLAG_RATIO and flags[1] == 0
    x, flags, _ = oracle_mod.solve_batch(-np.eye(2)[None], b[:1], method=1)
    assert flags[0] & oracle_mod.FLAG_SINGULAR


# ---------------------------------------------------------------- ALS loop
def test_exact_recovery_noiseless_full(oracle_mod):
    """Noiseless, fully observed rank-n_f R with lambda = 0: the U step fits
    R M (M^T M)^-1 exactly, so after one sweep U M^T reproduces R."""
    rng = np.random.default_rng(9)
    n_u, n_m, f = 30, 20, 4
    # Small integer factors keep R exactly representable in float32.
    U = rng.integers(-3, 4, (n_u, f)).astype(np.float64)
    M = rng.integers(-3, 4, (n_m, f)).astype(np.float64)
    assert np.linalg.matrix_rank(U) == f and np.linalg.matrix_rank(M) == f
    R = (U @ M.T).astype(np.float32)
    ii, jj = np.meshgrid(np.arange(n_u), np.arange(n_m), indexing="ij")
    rows = synth.coo_to_csr(ii.ravel(), jj.ravel(), R.ravel(), n_u, n_m)
    cols = synth.coo_to_csr(jj.ravel(), ii.ravel(), R.ravel(), n_m, n_u)
    M0 = rng.standard_normal((n_m, f))
    Uh, Mh = oracle_mod.fit(rows, cols, M0, 0.0, 1.0, 1, oracle_mod.GRAM_FULL)
    err = np.linalg.norm(Uh @ Mh.T - R.astype(np.float64)) / np.linalg.norm(R)
    assert err < 1e-10


def test_full_als_objective_non_increasing(oracle_mod):
    """Sec. 2.1: the objective of Eq. (object function) never increases."""
    p = synth.make_workload("small")
    lam = 0.1
    M = synth.init_factor(p.n_m, p.f, 1000).astype(np.float64)
    U = np.zeros((p.n_u, p.f))
    prev = np.inf
    R, Ct = p.train_rows, p.train_cols
    for _ in range(5):
        U, _, _ = oracle_mod.half_sweep(R.indptr, R.indices, R.values, M, lam, 1.0, oracle_mod.GRAM_FULL)
        o1 = oracle_mod.objective(R, Ct, U, M, lam)
        M, _, _ = oracle_mod.half_sweep(Ct.indptr, Ct.indices, Ct.values, U, lam, 1.0, oracle_mod.GRAM_FULL)
        o2 = oracle_mod.objective(R, Ct, U, M, lam)
        assert o1 <= prev * (1 + 1e-12) and o2 <= o1 * (1 + 1e-12)
        prev = o2


def test_objective_and_rmse_golden(oracle_mod):
    g = json.load(open(GOLDEN))["objective"]
    e = np.array(g["entries"])
    iu, im, r = e[:, 0].astype(np.int32), e[:, 1].astype(np.int32), e[:, 2].astype(np.float32)
    U, M = np.array(g["U"]), np.array(g["M"])
    rows = synth.coo_to_csr(iu, im, r, 2, 2)
    cols = synth.coo_to_csr(im, iu, r, 2, 2)
    assert oracle_mod.sse(iu, im, r, U, M) == g["sse"]
    assert oracle_mod.rmse(iu, im, r, U, M) == g["rmse"]
    assert oracle_mod.objective(rows, cols, U, M, g["lam"]) == pytest.approx(g["objective"], rel=1e-15)


def test_core_als_converges_on_small(oracle_mod):
    """Algorithm 2 on the 1000 x 500, n_f = 10 workload reaches a test RMSE
    close to full ALS (the paper's claim that CORE tracks FULL; a sanity
    check, not a pin)."""
    p = synth.make_workload("small")
    M0 = synth.init_factor(p.n_m, p.f, 1000)
    out = {}
    for name, r, mode in (("core", 0.5, oracle_mod.GRAM_ASYM), ("full", 1.0, oracle_mod.GRAM_FULL)):
        U, M = oracle_mod.fit(p.train_rows, p.train_cols, M0, 0.1, r, 10, mode)
        out[name] = oracle_mod.rmse(p.test_u, p.test_m, p.test_r, U, M)
    assert np.isfinite(out["core"]) and out["core"] < 3 * out["full"] + 0.5


# --------------------------------------------------------- Theorem 1 (soft)
@pytest.mark.parametrize("seed", range(10))
def test_theorem1_bound_when_hypothesis_holds(oracle_mod, seed):
    """Eq. (tm1): if ||M - M*||_2 <= eps' ||M||_2 with eps' below the stated
    bound, the core residual is within (1 + eps_m) of the full one. The
    smallest eps_m admitted by eps' is computed from the condition and the
    inequality is checked. Rows where c_m eps' >= 1 satisfy no eps_m and are
    skipped."""
    rng = np.random.default_rng(600 + seed)
    n, f, lam, budget = 40, 3, 0.05, 0.9
    X = rng.standard_normal((n, f))
    X[rng.random((n, f)) < 0.3] *= 1e-3  # numerically sparse design (Sec. 1)
    r = (X @ rng.standard_normal(f) + 0.3 * rng.standard_normal(n)).astype(np.float32)
    rr = r.astype(np.float64)
    s = oracle_mod.budget(n, budget)
    keep = oracle_mod.ces_row(X, s)
    Xs = X * keep
    indptr, idx, vals, Y = one_row_csr(X, r)
    xc, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, budget, oracle_mod.GRAM_ASYM)
    xf, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, 1.0, oracle_mod.GRAM_FULL)
    eps_p = np.linalg.norm(X - Xs, 2) / np.linalg.norm(X, 2)
    c_m = np.linalg.norm(X, 2) ** 2 * np.linalg.norm(np.linalg.inv(X.T @ X + lam * n * np.eye(f)), 2)
    rsse = np.linalg.norm(rr - X @ xf[0]) / np.linalg.norm(rr)
    if c_m * eps_p >= 1:
        pytest.skip("hypothesis of Theorem 1 admits no eps_m for this row")
    q = (c_m + 1) / (rsse * (1.0 / (c_m * eps_p) - 1.0))
    eps_m = (1 + q) ** 2 - 1
    lhs = np.linalg.norm(rr - X @ xc[0]) ** 2
    rhs = (1 + eps_m) * np.linalg.norm(rr - X @ xf[0]) ** 2
    assert lhs <= rhs * (1 + 1e-12)

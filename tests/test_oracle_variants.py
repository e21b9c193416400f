"""Pins of the oracle's variants and evaluation functions: the fixed
subsample size and the fast variant of Sec. 3, the objective with the plain
regulariser, the packed mask layout, ReMSE / P-ReMSE and the recommendation
metrics of Sec. 5.1.

As in test_oracle_pins.py, each check compares the oracle with an
independent route: brute force, Householder QR, reductions to an estimator
pinned elsewhere, hand-worked fixtures, or closed forms.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2509_18024_gb300 import synth
from test_oracle_pins import brute_force_keep, ridge_qr

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def csr_of(lengths, n_cols, rng):
    indptr = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=indptr[1:])
    idx = np.concatenate([np.sort(rng.choice(n_cols, size=int(L), replace=False)) for L in lengths]).astype(np.int32)
    vals = rng.standard_normal(int(indptr[-1])).astype(np.float32)
    return indptr, idx, vals


# ------------------------------------------------------ fixed subsample size
def test_fixed_budget_hand_values(oracle_mod):
    b = oracle_mod.budget
    assert b(10, 0.25, fixed_keep=3) == 3
    assert b(2, 0.25, fixed_keep=3) == 2
    assert b(0, 0.25, fixed_keep=3) == 0
    assert b(1000, 0.9, fixed_keep=7) == 7      # the rate is ignored
    assert b(10, 0.0, min_keep=5, fixed_keep=3) == 5
    assert b(4, 0.0, min_keep=5, fixed_keep=3) == 4


@pytest.mark.parametrize("seed", range(4))
def test_fixed_size_equals_rate_rule_row_by_row(oracle_mod, seed):
    """With s fixed, row i keeps min(n_i, s) per column, which is what the
    (pinned) rate rule keeps with r_i = (min(n_i, s) + 1/2) / n_i."""
    rng = np.random.default_rng(300 + seed)
    lengths = rng.integers(1, 30, 12)
    n_cols, f, s = 40, int(rng.integers(1, 6)), int(rng.integers(1, 9))
    indptr, idx, vals = csr_of(lengths, n_cols, rng)
    Y = rng.choice([-1.0, -0.5, 0.0, 0.5, 1.0, 2.0], size=(n_cols, f)) + 0.01 * rng.standard_normal((n_cols, f))
    lam = 0.1
    X, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, 0.0, fixed_keep=s)
    for i, n in enumerate(lengths):
        r_i = (min(int(n), s) + 0.5) / int(n)
        Xi, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, r_i, rows=[i])
        assert np.array_equal(X[i], Xi[i]), (seed, i)


def test_fixed_size_covering_every_row_is_full_als(oracle_mod):
    rng = np.random.default_rng(7)
    lengths = rng.integers(3, 25, 10)
    indptr, idx, vals = csr_of(lengths, 30, rng)
    Y = rng.standard_normal((30, 4))
    lam = 0.2
    X, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, 0.0, fixed_keep=int(lengths.max()))
    for i in range(len(lengths)):
        lo, hi = indptr[i], indptr[i + 1]
        ref = ridge_qr(Y[idx[lo:hi]], vals[lo:hi].astype(np.float64), lam * (hi - lo))
        np.testing.assert_allclose(X[i], ref, rtol=1e-10, atol=1e-12)


def test_fixed_size_masks_match_brute_force(oracle_mod):
    rng = np.random.default_rng(11)
    lengths = [1, 2, 5, 7]
    indptr, idx, _ = csr_of(lengths, 12, rng)
    Y = rng.choice([-2.0, -1.0, -0.0, 0.0, 1.0, 2.0], size=(12, 3))
    for s in range(0, 8):
        masks = oracle_mod.select_half(indptr, idx, Y, 0.0, fixed_keep=s)
        for i, n in enumerate(lengths):
            X = Y[idx[indptr[i]:indptr[i + 1]]]
            for a in range(3):
                ref = brute_force_keep(X[:, a], min(n, s)) if s > 0 else brute_force_keep(X[:, a], 0)
                got = (masks[indptr[i]:indptr[i + 1], 0] >> a) & 1
                assert np.array_equal(got, ref), (s, i, a)


# -------------------------------------------------------------- fast variant
def test_factor_sketch_matches_brute_force(oracle_mod):
    rng = np.random.default_rng(21)
    Y = rng.choice([-2.0, -1.0, -0.5, -0.0, 0.0, 0.5, 1.0, 2.0], size=(7, 4))
    for r in (0.0, 0.15, 0.3, 0.5, 0.9, 1.0):
        keep = oracle_mod.factor_sketch(Y, r)
        s = int(math.floor(7 * r))
        for a in range(4):
            assert np.array_equal(keep[:, a], brute_force_keep(Y[:, a], s)), (r, a)


@pytest.mark.parametrize("gram", [0, 1])
def test_fast_variant_on_fully_observed_rows_is_algorithm_2(oracle_mod, gram):
    """When every row observes every column, a row's slice is the whole
    factor in index order: the factor-wide CES is the slice's own CES."""
    rng = np.random.default_rng(31 + gram)
    n_rows, n_cols, f = 6, 25, 5
    indptr = np.arange(n_rows + 1, dtype=np.int64) * n_cols
    idx = np.tile(np.arange(n_cols, dtype=np.int32), n_rows)
    vals = rng.standard_normal(n_rows * n_cols).astype(np.float32)
    Y = rng.choice([-1.0, 1.0, 0.5, -0.5, 2.0], size=(n_cols, f)) * (1 + 0.1 * rng.random((n_cols, f)))
    for r in (0.2, 0.36, 0.6):
        Xs, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, 0.1, r, gram, sketch="slice")
        Xf, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, 0.1, r, gram, sketch="factor")
        assert np.array_equal(Xs, Xf), r


@pytest.mark.parametrize("seed", range(3))
def test_fast_variant_row_subset_reduction(oracle_mod, seed):
    """Rows K of the factor dominate every column (|y| in [5, 6] against
    [0, 1]) and s = floor(n_other r) = |K|: the factor-wide sketch keeps K in
    every column, so X*^T X is X_J^T X_J over J = I_i & K and the estimator
    is ridge least squares on J with penalty lambda n_i (n_i the full count)."""
    rng = np.random.default_rng(40 + seed)
    n_cols, f = 50, 4
    K = np.sort(rng.choice(n_cols, size=10, replace=False))
    Y = rng.uniform(0.0, 1.0, (n_cols, f)) * rng.choice([-1, 1], (n_cols, f))
    Y[K] = rng.uniform(5.0, 6.0, (len(K), f)) * rng.choice([-1, 1], (len(K), f))
    r = 10.5 / n_cols
    lengths = rng.integers(15, 40, 8)
    indptr, idx, vals = csr_of(lengths, n_cols, rng)
    lam = 0.05
    X, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, lam, r, sketch="factor")
    for i in range(len(lengths)):
        lo, hi = indptr[i], indptr[i + 1]
        sel = np.isin(idx[lo:hi], K)
        ref = ridge_qr(Y[idx[lo:hi][sel]], vals[lo:hi][sel].astype(np.float64), lam * (hi - lo))
        np.testing.assert_allclose(X[i], ref, rtol=1e-10, atol=1e-12)


def test_fast_variant_full_budget_is_full_als(oracle_mod):
    rng = np.random.default_rng(51)
    indptr, idx, vals = csr_of(rng.integers(2, 20, 9), 30, rng)
    Y = rng.standard_normal((30, 3))
    X, _, _ = oracle_mod.half_sweep(indptr, idx, vals, Y, 0.1, 1.0, sketch="factor")
    for i in range(9):
        lo, hi = indptr[i], indptr[i + 1]
        ref = ridge_qr(Y[idx[lo:hi]], vals[lo:hi].astype(np.float64), 0.1 * (hi - lo))
        np.testing.assert_allclose(X[i], ref, rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------- mask packing
def test_mask_packing_two_words_golden(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "mask_packing_f40.json")))
    f = g["n_f"]
    X = np.ones((2, f))
    for a in range(f):
        if a < 36:
            X[a % 2, a] = 2.0
        else:
            X[:, a] = 3.0
    masks = oracle_mod.select_half(np.array([0, 2], np.int64), np.array([0, 1], np.int32), X, g["budget"])
    assert masks.dtype == np.uint32 and masks.shape == (2, 2)
    assert masks.tolist() == g["masks"]


# ---------------------------------------------------------------- objective
def test_objective_plain_regulariser_hand_value(oracle_mod):
    # R (2 x 2) observed at (0,0)=1, (0,1)=2, (1,1)=3; f = 1, U = [1, 2], M = [0.5, 1].
    rows = synth.CSR(2, 2, np.array([0, 2, 3], np.int64), np.array([0, 1, 1], np.int32),
                     np.array([1.0, 2.0, 3.0], np.float32))
    cols = synth.CSR(2, 2, np.array([0, 1, 3], np.int64), np.array([0, 0, 1], np.int32),
                     np.array([1.0, 2.0, 3.0], np.float32))
    U = np.array([[1.0], [2.0]])
    M = np.array([[0.5], [1.0]])
    # residuals 0.5, 1, 1 -> 2.25; plain penalty 0.1 (1 + 4 + 0.25 + 1) = 0.625;
    # weighted 0.1 (2*1 + 1*4 + 1*0.25 + 2*1) = 0.825.
    assert oracle_mod.objective(rows, cols, U, M, 0.1, oracle_mod.REG_PLAIN) == pytest.approx(2.875, abs=1e-14)
    assert oracle_mod.objective(rows, cols, U, M, 0.1) == pytest.approx(3.075, abs=1e-14)


# ------------------------------------------------------------ ReMSE / P-ReMSE
def test_remse_hand_values(oracle_mod):
    iu = np.array([0, 1], np.int32)
    im = np.array([0, 0], np.int32)
    r = np.array([3.0, 4.0], np.float32)
    U = np.array([[1.0], [0.0]])
    M = np.array([[3.0]])
    assert oracle_mod.remse(iu, im, r, U, M) == pytest.approx(0.8, abs=1e-15)  # sqrt(16) / sqrt(25)
    assert oracle_mod.remse(iu, im, r, np.zeros((2, 1)), M) == pytest.approx(1.0, abs=1e-15)
    U2 = np.array([[1.0], [4.0 / 3.0]])
    assert oracle_mod.remse(iu, im, r, U2, M) < 1e-15
    assert math.isnan(oracle_mod.remse(iu[:0], im[:0], r[:0], U, M))


# ------------------------------------------------------ recommendation metrics
def _csr_lists(lists):
    indptr = np.zeros(len(lists) + 1, np.int64)
    np.cumsum([len(x) for x in lists], out=indptr[1:])
    idx = np.array([j for x in lists for j in sorted(x)], np.int32)
    return indptr, idx


def test_ranking_golden(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "ranking_small.json")))
    U = np.array(g["U"], np.float32)
    M = np.array(g["M"], np.float32)
    tip, tix = _csr_lists(g["train"])
    rip, rix = _csr_lists(g["relevant"])
    top = oracle_mod.rank_topk(U, M, tip, tix, g["K"])
    assert top.tolist() == g["topk"]
    h1, _, n = oracle_mod.rank_metrics(top, rip, rix, k_hit=1, k_ndcg=3)
    h2, ndcg3, _ = oracle_mod.rank_metrics(top, rip, rix, k_hit=2, k_ndcg=3)
    assert n == g["n_eval"]
    assert h1 == g["hit_at_1"] and h2 == g["hit_at_2"]
    l3 = math.log2(3.0)
    assert ndcg3 == pytest.approx((1 / l3 + 0.5 / (1 + 1 / l3)) / 2, abs=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_ranking_matches_brute_force_on_exact_scores(oracle_mod, seed):
    """Small-integer factors make every predicted rating exact in FP32, so a
    plain sort of the exact scores (numpy lexsort, ties to the lower item)
    must give the same lists; ties are frequent by construction."""
    rng = np.random.default_rng(60 + seed)
    n_u, n_m, f, K = 30, 40, 3, 10
    U = rng.integers(-2, 3, (n_u, f)).astype(np.float32)
    M = rng.integers(-2, 3, (n_m, f)).astype(np.float32)
    train = [sorted(rng.choice(n_m, size=int(rng.integers(0, 35)), replace=False).tolist()) for _ in range(n_u)]
    tip, tix = _csr_lists(train)
    top = oracle_mod.rank_topk(U, M, tip, tix, K)
    scores = U.astype(np.int64) @ M.astype(np.int64).T
    for i in range(n_u):
        cand = np.array([j for j in range(n_m) if j not in set(train[i])], np.int64)
        order = cand[np.lexsort((cand, -scores[i, cand]))] if cand.size else cand
        want = list(order[:K]) + [-1] * max(0, K - len(order))
        assert top[i].tolist() == want, i


def test_ranking_all_relevant_scores_one(oracle_mod):
    rng = np.random.default_rng(70)
    U = rng.standard_normal((20, 4)).astype(np.float32)
    M = rng.standard_normal((15, 4)).astype(np.float32)
    tip, tix = _csr_lists([[] for _ in range(20)])
    top = oracle_mod.rank_topk(U, M, tip, tix, 10)
    rip, rix = _csr_lists([list(range(15)) for _ in range(20)])
    hit, ndcg, n = oracle_mod.rank_metrics(top, rip, rix, 5, 10)
    assert (hit, n) == (1.0, 20)
    assert ndcg == pytest.approx(1.0, abs=1e-15)
    # No relevant item in any list: both metrics are 0.
    rip0, rix0 = _csr_lists([[j for j in range(15) if j not in top[i]] for i in range(20)])
    hit0, ndcg0, _ = oracle_mod.rank_metrics(top, rip0, rix0, 5, 10)
    assert hit0 == 0.0 and ndcg0 == 0.0


# ---------------------------------------------------------------- simulation
def test_simulation_design_shapes():
    p = synth.simulation("D2", 0.7, n_u=60, n_m=50, f=6, seed=3)
    assert p.train_rows.nnz + len(p.pred_r) == 60 * 50
    assert len(p.pred_r) == round(0.7 * 3000)
    assert (p.U_true > 0).all()  # log-normal factors
    cells = set(zip(p.pred_u.tolist(), p.pred_m.tolist()))
    rows = np.repeat(np.arange(60), np.diff(p.train_rows.indptr))
    assert not cells & set(zip(rows.tolist(), p.train_rows.indices.tolist()))

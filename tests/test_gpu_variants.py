"""Parity of the CUDA path with the FP64 oracle for the variants of Sec. 3 and
the evaluation calls.

* Fixed subsample size (s_i = min(n_i, s)) and the fast variant (CES once on
  the whole design factor): masks bit-exact, one half-sweep from identical
  FP32 inputs within 1e-5 relative Frobenius error, across every row bucket
  (warp rows, CTA-resident rows, split rows) and the CUDA-core and
  tensor-core widths; a full fit's test RMSE within 1e-3 of the oracle's.
* The objective of Eq. (object function) on the GPU equals the oracle's on the
  same factors (1e-6 relative: FP32 predictions), and full ALS does not increase it across GPU
  half-sweeps (Sec. 2.1).
* ReMSE / P-ReMSE on the simulation design of Sec. 5.1 equal the oracle's on
  the same factors; recommendation lists bit-exact and Hit@5 / NDCG@10 equal
  the oracle's (1e-12).
"""
import numpy as np
import pytest

import oracle
from paper_2509_18024_gb300 import synth
from tests.helpers import rel_fro, rows_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALF_TOL = 1e-5
LENGTHS = [0, 1, 2, 3, 5, 8, 31, 32, 33, 64, 100, 255, 256, 257, 511, 513, 1000, 1025, 3000, 9000]


@pytest.fixture(scope="module")
def core():
    from paper_2509_18024_gb300 import core_als
    return core_als


def f32(x):
    return float(np.float32(x))


def check_variant(core, csr, Y, f, lam, r, mode="asym", fixed_keep=0, sketch="slice", precision=0, tol=HALF_TOL):
    gm = {"asym": oracle.GRAM_ASYM, "sym": oracle.GRAM_SYM, "full": oracle.GRAM_FULL}[mode]
    eng = core.CoreALS(f, f32(lam), r, gram_mode=mode, fixed_keep=fixed_keep, sketch=sketch, precision=precision)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    X = eng.half_sweep(R, Yd).cpu().numpy()
    masks = eng.select(R, Yd).cpu().numpy().view(np.uint32)
    Y64 = Y.astype(np.float64)
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y64, f32(lam), r, gm, fixed_keep=fixed_keep,
                                 sketch=sketch)
    if mode != "full":
        mo = oracle.select_half(csr.indptr, csr.indices, Y64, r, fixed_keep=fixed_keep, sketch=sketch)
        bad = np.nonzero(masks != mo)[0]
        assert bad.size == 0, f"{bad.size} mask words differ, first entries {bad[:5]}"
    err = rel_fro(X, Xo)
    assert err <= tol, f"rel Frobenius {err:.3e} (f={f}, {mode}, fixed={fixed_keep}, {sketch}, prec={precision})"
    return err


# ------------------------------------------------------ fixed subsample size
@pytest.mark.parametrize("f", [10, 32])
@pytest.mark.parametrize("s", [1, 8, 40, 5000])
def test_fixed_size_half_sweep(core, f, s):
    csr, Y = rows_problem(LENGTHS, 12000, f, seed=100 + s)
    check_variant(core, csr, Y, f, 0.05, 0.25, "asym", fixed_keep=s)
    check_variant(core, csr, Y, f, 0.05, 0.25, "sym", fixed_keep=s)


def test_fixed_size_wide_tensor_core(core):
    csr, Y = rows_problem(LENGTHS, 12000, 64, seed=7)
    check_variant(core, csr, Y, 64, 0.05, 0.25, "asym", fixed_keep=24)


# ------------------------------------------------------------- fast variant
@pytest.mark.parametrize("f", [1, 8, 10, 16, 32])
@pytest.mark.parametrize("r", [0.1, 0.25, 0.5])
def test_fast_variant_half_sweep(core, f, r):
    csr, Y = rows_problem(LENGTHS, 12000, f, seed=200 + f)
    check_variant(core, csr, Y, f, 0.05, r, "asym", sketch="factor")


@pytest.mark.parametrize("mode", ["sym", "full"])
def test_fast_variant_other_modes(core, mode):
    csr, Y = rows_problem(LENGTHS, 12000, 32, seed=17)
    check_variant(core, csr, Y, 32, 0.05, 1.0 if mode == "full" else 0.3, mode, sketch="factor")


def test_fast_variant_ties(core):
    pool = [0.0, -0.0, 0.5, -0.5, 1.0, -1.0, 0.25]
    csr, Y = rows_problem(LENGTHS, 12000, 32, seed=5, pool=pool)
    for r in (0.1, 0.25, 0.5):
        eng = core.CoreALS(32, 0.05, r, sketch="factor")
        masks = eng.select(core.DeviceCSR.from_host(csr), torch.as_tensor(Y).cuda()).cpu().numpy().view(np.uint32)
        mo = oracle.select_half(csr.indptr, csr.indices, Y.astype(np.float64), r, sketch="factor")
        assert np.array_equal(masks, mo), r


@pytest.mark.parametrize("f,prec", [(64, 0), (128, 0), (64, 1)])
def test_fast_variant_wide(core, f, prec):
    csr, Y = rows_problem(LENGTHS, 12000, f, seed=300 + f)
    tol = HALF_TOL if prec == 0 else 1e-3
    check_variant(core, csr, Y, f, 0.05, 0.25, "asym", sketch="factor", precision=prec, tol=tol)


@pytest.mark.parametrize("variant", [dict(sketch="factor"), dict(fixed_keep=6)])
def test_variant_fit_rmse_matches_oracle(core, variant):
    p = synth.make_workload("small")
    M0 = synth.init_factor(p.n_m, p.f, 1000)
    eng = core.CoreALS(p.f, f32(0.1), 0.5, **variant)
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    test = tuple(torch.as_tensor(a).cuda() for a in (p.test_u, p.test_m, p.test_r))
    _, _, rep = eng.fit(Ru, Ri, torch.as_tensor(M0).cuda(), 10, test=test)
    Uo, Mo = oracle.fit(p.train_rows, p.train_cols, M0, f32(0.1), 0.5, 10, **variant)
    ro = oracle.rmse(p.test_u, p.test_m, p.test_r, Uo, Mo)
    assert abs(rep["test_rmse"] - ro) <= 1e-3 * ro, (variant, rep["test_rmse"], ro)


# ---------------------------------------------------------------- objective
@pytest.mark.parametrize("reg", ["weighted", "plain"])
def test_objective_matches_oracle(core, reg):
    p = synth.make_workload("small")
    M0 = synth.init_factor(p.n_m, p.f, 1000)
    lam = f32(0.1)
    eng = core.CoreALS(p.f, lam, 0.5, reg_mode=reg)
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    U, M, rep = eng.fit(Ru, Ri, torch.as_tensor(M0).cuda(), 3)
    Uh, Mh = U.cpu().numpy(), M.cpu().numpy()
    ref = oracle.objective(p.train_rows, p.train_cols, Uh, Mh, lam,
                           oracle.REG_PLAIN if reg == "plain" else oracle.REG_WEIGHTED)
    # The GPU predicts in FP32 (sums in FP64): each prediction is off by at
    # most about f 2^-24 of sum_a |u_a m_a|, so the data term by at most
    # 2 f 2^-24 sum_e |res_e| sum_a |u_a m_a|, below 1e-6 of f here.
    assert rep["objective"] == pytest.approx(ref, rel=1e-6)
    assert eng.objective(Ru, Ri, U, M) == rep["objective"]


def test_full_als_objective_does_not_increase_on_the_gpu(core):
    p = synth.make_workload("small")
    lam = f32(0.1)
    eng = core.CoreALS(p.f, lam, 1.0, gram_mode="full")
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    M = torch.as_tensor(synth.init_factor(p.n_m, p.f, 1000)).cuda()
    U = eng.half_sweep(Ru, M)
    prev = eng.objective(Ru, Ri, U, M)
    for _ in range(8):
        for R, Y, X in ((Ri, U, M), (Ru, M, U)):
            eng.half_sweep(R, Y, X)
            cur = eng.objective(Ru, Ri, U, M)
            # Each half-sweep minimises f exactly over one side (FP32 solve):
            # allow FP32-level slack only.
            assert cur <= prev * (1 + 1e-6), (cur, prev)
            prev = cur


# ------------------------------------------------- Sec. 5.1 evaluation calls
@pytest.fixture(scope="module")
def sim():
    return synth.simulation("D1", 0.6, n_u=600, n_m=500, f=60, seed=4)


def test_remse_on_the_simulation_design(core, sim):
    p = sim
    eng = core.CoreALS(p.f, f32(0.05), 0.2)
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    M0 = torch.as_tensor(synth.init_factor(p.n_m, p.f, 9)).cuda()
    U, M, _ = eng.fit(Ru, Ri, M0, 4)
    Uh, Mh = U.cpu().numpy(), M.cpu().numpy()
    rows = np.repeat(np.arange(p.n_u, dtype=np.int32), np.diff(p.train_rows.indptr))
    emp = (rows, p.train_rows.indices, p.train_rows.values)
    pred = (p.pred_u, p.pred_m, p.pred_r)
    for iu, im, r in (emp, pred):
        got = eng.remse(*(torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in (iu, im, r)), U, M)
        assert got == pytest.approx(oracle.remse(iu, im, r, Uh, Mh), rel=1e-6)


@pytest.mark.parametrize("f", [10, 32, 60])
def test_ranking_lists_and_metrics_match_oracle(core, f):
    p = synth.simulation("D3", 0.5, n_u=400, n_m=700, f=f, seed=f)
    rng = np.random.default_rng(f)
    U = (rng.standard_normal((p.n_u, f)) * 0.3).astype(np.float32)
    M = (rng.standard_normal((p.n_m, f)) * 0.3).astype(np.float32)
    rel = synth.relevant_items(p.n_u, p.n_m, p.pred_u, p.pred_m, p.pred_r, synth.top_share_threshold(p.pred_r))
    eng = core.CoreALS(f, 0.05, 0.25)
    Rt = core.DeviceCSR.from_host(p.train_rows)
    Rr = core.DeviceCSR.from_host(rel)
    hit, ndcg, n, lists = eng.ranking(Rt, Rr, torch.as_tensor(U).cuda(), torch.as_tensor(M).cuda(), 5, 10,
                                      want_lists=True)
    top = oracle.rank_topk(U, M, p.train_rows.indptr, p.train_rows.indices, 10)
    assert np.array_equal(lists.cpu().numpy(), top)
    ho, no, nn = oracle.rank_metrics(top, rel.indptr, rel.indices, 5, 10)
    assert n == nn
    assert hit == pytest.approx(ho, abs=1e-12) and ndcg == pytest.approx(no, abs=1e-12)


def test_ranking_ties_and_short_lists(core):
    # Integer factors: many exact ties in the predicted ratings; a user who
    # rated all but 3 items gets a list padded with -1.
    rng = np.random.default_rng(3)
    n_u, n_m, f = 50, 40, 3
    U = rng.integers(-2, 3, (n_u, f)).astype(np.float32)
    M = rng.integers(-2, 3, (n_m, f)).astype(np.float32)
    train = [sorted(rng.choice(n_m, size=int(rng.integers(0, 30)), replace=False).tolist()) for _ in range(n_u)]
    train[0] = list(range(37))
    ip = np.zeros(n_u + 1, np.int64)
    np.cumsum([len(t) for t in train], out=ip[1:])
    ix = np.array([j for t in train for j in t], np.int32)
    Rt = synth.CSR(n_u, n_m, ip, ix, np.ones(len(ix), np.float32))
    rel = synth.CSR(n_u, n_m, np.arange(n_u + 1, dtype=np.int64), (np.arange(n_u) % n_m).astype(np.int32),
                    np.ones(n_u, np.float32))
    eng = core.CoreALS(f, 0.05, 0.25)
    hit, ndcg, n, lists = eng.ranking(core.DeviceCSR.from_host(Rt), core.DeviceCSR.from_host(rel),
                                      torch.as_tensor(U).cuda(), torch.as_tensor(M).cuda(), 5, 10, want_lists=True)
    top = oracle.rank_topk(U, M, ip, ix, 10)
    assert np.array_equal(lists.cpu().numpy(), top)
    assert (top[0, 3:] == -1).all()
    ho, no, _ = oracle.rank_metrics(top, rel.indptr, rel.indices, 5, 10)
    assert hit == pytest.approx(ho, abs=1e-12) and ndcg == pytest.approx(no, abs=1e-12)


# ------------------------------------- the benchmark's full workload, sampled
@pytest.fixture(scope="module")
def zipf():
    return synth.make_workload("zipf_100k")


@pytest.mark.parametrize("variant", [dict(sketch="factor"), dict(fixed_keep=16)])
@pytest.mark.parametrize("side", ["users", "items"])
def test_variants_full_size_sampled_rows(core, zipf, variant, side):
    """The 100k x 20k, 10M-entry, n_f = 32 workload: every row on the GPU in
    the benchmark's launch configuration, a sample of rows (the longest ones
    included) against the oracle, masks bit-exact on the sample."""
    f, lam, r = 32, f32(0.05), 0.25
    if side == "users":
        csr, Y = zipf.train_rows, synth.init_factor(zipf.n_m, f, 1000)
    else:
        csr, Y = zipf.train_cols, synth.init_factor(zipf.n_u, f, 2000)
    eng = core.CoreALS(f, lam, r, **variant)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    X = eng.half_sweep(R, Yd).cpu().numpy()
    masks = eng.select(R, Yd).cpu().numpy().view(np.uint32)
    L = np.diff(csr.indptr)
    rng = np.random.default_rng(1)
    sample = np.unique(np.concatenate([np.argsort(L)[-12:], rng.choice(csr.n_rows, 300, replace=False)]))
    Y64 = Y.astype(np.float64)
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y64, lam, r, rows=sample, **variant)
    assert rel_fro(X[sample], Xo[sample]) <= HALF_TOL
    lens = L[sample]
    sub_ptr = np.zeros(len(sample) + 1, np.int64)
    np.cumsum(lens, out=sub_ptr[1:])
    take = np.concatenate([np.arange(csr.indptr[i], csr.indptr[i + 1]) for i in sample])
    mo = oracle.select_half(sub_ptr, csr.indices[take], Y64, r, **variant)
    assert np.array_equal(masks[take], mo)


def test_objective_and_ranking_full_size(core, zipf):
    """Eq. (object function) over the 9M training entries, and the ranked
    lists of 100k users over 20k items (ratings >= 4 of the held-out set as
    the relevant items, Sec. 6's rule for rating data): the objective equals
    the oracle's within the FP32-prediction bound, the lists of sampled users
    bit-exact, and Hit@5 / NDCG@10 of those users equal the oracle's."""
    f, lam = 32, f32(0.05)
    rng = np.random.default_rng(5)
    U = (rng.standard_normal((zipf.n_u, f)) * 0.4).astype(np.float32)
    M = (rng.standard_normal((zipf.n_m, f)) * 0.4).astype(np.float32)
    eng = core.CoreALS(f, lam, 0.25)
    Ru = core.DeviceCSR.from_host(zipf.train_rows)
    Ri = core.DeviceCSR.from_host(zipf.train_cols)
    Ud, Md = torch.as_tensor(U).cuda(), torch.as_tensor(M).cuda()
    obj = eng.objective(Ru, Ri, Ud, Md)
    assert obj == pytest.approx(oracle.objective(zipf.train_rows, zipf.train_cols, U, M, lam), rel=1e-6)
    rel = synth.relevant_items(zipf.n_u, zipf.n_m, zipf.test_u, zipf.test_m, zipf.test_r, 4.0)
    hit, ndcg, n, lists = eng.ranking(Ru, core.DeviceCSR.from_host(rel), Ud, Md, 5, 10, want_lists=True)
    lists = lists.cpu().numpy()
    users = np.sort(rng.choice(zipf.n_u, 300, replace=False))
    ip = zipf.train_rows.indptr
    sub_ip = np.concatenate([[0], np.cumsum(np.diff(ip)[users])]).astype(np.int64)
    sub_ix = np.concatenate([zipf.train_rows.indices[ip[u]:ip[u + 1]] for u in users])
    top = oracle.rank_topk(U[users], M, sub_ip, sub_ix, 10)
    assert np.array_equal(lists[users], top)
    rip = rel.indptr
    sub_rp = np.concatenate([[0], np.cumsum(np.diff(rip)[users])]).astype(np.int64)
    sub_rx = np.concatenate([rel.indices[rip[u]:rip[u + 1]] for u in users]).astype(np.int32)
    ho, no, _ = oracle.rank_metrics(lists[users], sub_rp, sub_rx, 5, 10)
    ho2, no2, _ = oracle.rank_metrics(top, sub_rp, sub_rx, 5, 10)
    assert (ho, no) == (ho2, no2)
    assert n == int((np.diff(rip) > 0).sum())
    # The metrics over all users equal the oracle's on the GPU's lists (whose
    # sampled rows were just checked).
    ha, na, nn = oracle.rank_metrics(lists, rel.indptr, rel.indices, 5, 10)
    assert nn == n and hit == pytest.approx(ha, abs=1e-12) and ndcg == pytest.approx(na, abs=1e-12)

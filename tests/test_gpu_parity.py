"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: CES masks bit-exact; one half-sweep from identical FP32 input factors
within 1e-5 relative Frobenius error (FP32 path); assembled systems within
1e-5 relative per row; the final test RMSE of a full run within 1e-3
relative.
"""
import numpy as np
import pytest

import oracle
from paper_2509_18024_gb300 import synth
from tests.helpers import rel_fro, rows_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HALF_TOL = 1e-5
MODES = {"asym": oracle.GRAM_ASYM, "sym": oracle.GRAM_SYM, "full": oracle.GRAM_FULL}


@pytest.fixture(scope="module")
def core():
    from paper_2509_18024_gb300 import core_als
    return core_als


@pytest.fixture(scope="module")
def small():
    return synth.make_workload("small")


def f32(x):
    return float(np.float32(x))


def gpu_half(core, csr, Y, f, lam, r, mode="asym", reg="weighted", min_keep=0):
    eng = core.CoreALS(f, lam, r, gram_mode=mode, reg_mode=reg, min_keep=min_keep)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    flags = torch.zeros(csr.n_rows, dtype=torch.int32, device="cuda")
    X = eng.half_sweep(R, Yd, flags=flags)
    masks = eng.select(R, Yd)
    torch.cuda.synchronize()
    out = X.cpu().numpy(), flags.cpu().numpy(), masks.cpu().numpy().view(np.uint32), eng
    return out


def oracle_half(csr, Y, lam, r, mode="asym", reg="weighted", min_keep=0, rows=None):
    return oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), f32(lam), r,
                             MODES[mode], oracle.REG_PLAIN if reg == "plain" else oracle.REG_WEIGHTED,
                             min_keep, rows=rows)


def check_half(core, csr, Y, f, lam, r, mode="asym", reg="weighted", min_keep=0, tol=HALF_TOL):
    X, flags, masks, _ = gpu_half(core, csr, Y, f, lam, r, mode, reg, min_keep)
    Xo, fo, _ = oracle_half(csr, Y, lam, r, mode, reg, min_keep)
    mo = oracle.select_half(csr.indptr, csr.indices, Y.astype(np.float64), 1.0 if mode == "full" else r,
                            min_keep)
    bad = np.nonzero(masks != mo)[0]
    assert bad.size == 0, f"{bad.size} mask words differ, first entries {bad[:5]}"
    err = rel_fro(X, Xo)
    rowerr = np.linalg.norm(X - Xo, axis=1) / np.maximum(np.linalg.norm(Xo, axis=1), 1e-30)
    worst = int(np.argmax(rowerr)) if rowerr.size else -1
    assert err <= tol, (f"rel Frobenius {err:.3e} > {tol:.0e}; worst row {worst} "
                        f"len {csr.indptr[worst + 1] - csr.indptr[worst]} err {rowerr[worst]:.3e}")
    # Flags agree on singular rows (those are exactly decided).
    assert np.array_equal(flags & 2, fo & 2)
    return err


# ------------------------------------------------------------ small workload
@pytest.mark.parametrize("mode,r", [("asym", 0.5), ("asym", 0.25), ("asym", 0.1), ("asym", 1.0),
                                    ("sym", 0.5), ("full", 1.0)])
def test_user_half_sweep_small(core, small, mode, r):
    M0 = synth.init_factor(small.n_m, small.f, 1000)
    check_half(core, small.train_rows, M0, small.f, 0.1, r, mode)


def test_item_half_sweep_small(core, small):
    M0 = synth.init_factor(small.n_m, small.f, 1000)
    U, _, _ = oracle_half(small.train_rows, M0, 0.1, 0.5)
    check_half(core, small.train_cols, U.astype(np.float32), small.f, 0.1, 0.5)


def test_plain_regulariser_and_min_keep(core, small):
    M0 = synth.init_factor(small.n_m, small.f, 1001)
    check_half(core, small.train_rows, M0, small.f, 1.0, 0.25, reg="plain")
    check_half(core, small.train_rows, M0, small.f, 0.1, 0.1, min_keep=3)


def test_ill_conditioned_rows_meet_fp32_perturbation_bound(core, small):
    """Plain lambda = 0.1 with r = 0.25 leaves rows whose system has
    condition number ~5e4: storing that system in FP32 alone moves the
    solution by ~kappa * 2^-24. Each row must stay within the first-order
    perturbation bound kappa(G) (|dG|/|G| + |db|/|b|) with both relative
    perturbations taken as (n_i + n_f) * 2^-24 (FP32 accumulation of n_i
    products and the elimination)."""
    M0 = synth.init_factor(small.n_m, small.f, 1001)
    csr = small.train_rows
    lam, r = 0.1, 0.25
    X, _, masks, _ = gpu_half(core, csr, M0, small.f, lam, r, reg="plain")
    Xo, _, _ = oracle_half(csr, M0, lam, r, reg="plain")
    G, b = oracle.assemble_half(csr.indptr, csr.indices, csr.values, M0.astype(np.float64), f32(lam), r,
                                oracle.GRAM_ASYM, oracle.REG_PLAIN)
    u = 2.0 ** -24
    L = np.diff(csr.indptr)
    worst = 0.0
    for i in range(csr.n_rows):
        nx = np.linalg.norm(Xo[i])
        if nx == 0:
            continue
        kappa = np.linalg.cond(G[i])
        bound = kappa * 2 * (L[i] + small.f) * u
        err = np.linalg.norm(X[i] - Xo[i]) / nx
        worst = max(worst, err / bound)
        assert err <= bound, (i, err, bound, kappa)
    assert worst > 0


# ------------------------------------------------------------------ ragged
LENGTHS = [0, 1, 2, 3, 5, 8, 31, 32, 33, 64, 100, 255, 256, 257, 511, 513, 1000, 3000]


@pytest.mark.parametrize("f", [1, 7, 8, 10, 16, 17, 32])
def test_ragged_rows_all_widths(core, f):
    csr, Y = rows_problem(LENGTHS, 4000, f, seed=f)
    for mode, r in (("asym", 0.25), ("sym", 0.5), ("full", 1.0)):
        check_half(core, csr, Y, f, 0.05, r, mode)


@pytest.mark.parametrize("r", [0.0, 0.1, 0.29, 0.5, 0.9, 1.0])
def test_budget_edges(core, r):
    csr, Y = rows_problem(LENGTHS, 4000, 32, seed=11)
    check_half(core, csr, Y, 32, 0.05, r, "asym")


def test_ties_zeros_and_signed_zero(core):
    # Y drawn from a tiny set: most comparisons are ties, resolved by position.
    pool = [0.0, -0.0, 0.5, -0.5, 1.0, -1.0, 0.25]
    csr, Y = rows_problem(LENGTHS, 4000, 32, seed=5, pool=pool)
    for r in (0.1, 0.25, 0.5, 0.75):
        X, _, masks, _ = gpu_half(core, csr, Y, 32, 0.05, r)
        mo = oracle.select_half(csr.indptr, csr.indices, Y.astype(np.float64), r)
        assert np.array_equal(masks, mo), f"masks differ at r={r}"


def test_long_rows_streamed(core):
    csr, Y = rows_problem([20000, 4097, 40000], 50000, 32, seed=3)
    for r in (0.1, 0.25, 0.5):
        check_half(core, csr, Y, 32, 0.05, r, "asym")
    check_half(core, csr, Y, 32, 0.05, 1.0, "full")


# ------------------------------------------------------ assemble and solve
@pytest.mark.parametrize("mode", ["asym", "sym", "full"])
def test_assemble_matches_oracle(core, mode):
    csr, Y = rows_problem(LENGTHS, 4000, 16, seed=21)
    eng = core.CoreALS(16, f32(0.05), 0.25, gram_mode=mode)
    G, b = eng.assemble(core.DeviceCSR.from_host(csr), torch.as_tensor(Y).cuda())
    Go, bo = oracle.assemble_half(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), f32(0.05), 0.25,
                                  MODES[mode])
    G, b = G.cpu().numpy(), b.cpu().numpy()
    for i in range(csr.n_rows):
        scale = max(np.abs(Go[i]).max(), 1e-30)
        assert np.abs(G[i] - Go[i]).max() <= 1e-5 * scale, i
        bs = max(np.abs(bo[i]).max(), 1e-30)
        assert np.abs(b[i] - bo[i]).max() <= 1e-5 * bs + 1e-30, i


@pytest.mark.parametrize("mode", ["asym", "sym"])
def test_solve_matches_oracle(core, mode):
    rng = np.random.default_rng(8)
    n, f = 500, 24
    A = rng.standard_normal((n, f, f)).astype(np.float32)
    if mode == "sym":
        A = (A @ np.transpose(A, (0, 2, 1)) + f * np.eye(f)).astype(np.float32)
    else:
        A = (A + 6 * np.eye(f)).astype(np.float32)
    b = rng.standard_normal((n, f)).astype(np.float32)
    eng = core.CoreALS(f, 0.05, 0.25, gram_mode=mode)
    X, flags = eng.solve(torch.as_tensor(A).cuda(), torch.as_tensor(b).cuda())
    Xo, fo, _ = oracle.solve_batch(A.astype(np.float64), b.astype(np.float64), 0 if mode == "asym" else 1)
    assert rel_fro(X.cpu().numpy(), Xo) <= 1e-4
    assert np.array_equal(flags.cpu().numpy(), fo)


def test_solve_flags_singular_and_ratio(core):
    f = 4
    G = np.stack([np.zeros((f, f)), np.diag([1.0, 1.0, 1.0, 1e-8]), np.eye(f)]).astype(np.float32)
    b = np.ones((3, f), np.float32)
    eng = core.CoreALS(f, 0.05, 0.25)
    X, flags = eng.solve(torch.as_tensor(G).cuda(), torch.as_tensor(b).cuda())
    flags = flags.cpu().numpy()
    assert flags[0] & 2 and np.all(X.cpu().numpy()[0] == 0)
    assert flags[1] == 1 and flags[2] == 0


@pytest.mark.parametrize("mode", ["asym", "sym"])
def test_solve_padded_odd_count_with_bad_systems(core, mode):
    # n_f = 30 pads to 32 (two identity rows per system); an odd count of
    # systems, with singular (all-zero) systems at an even and at the last
    # position and a near-singular one at an odd position.
    rng = np.random.default_rng(9)
    n, f = 9, 30
    A = rng.standard_normal((n, f, f))
    if mode == "sym":
        A = A @ np.transpose(A, (0, 2, 1)) + f * np.eye(f)
    else:
        A = A + 6 * np.eye(f)
    A[2] = 0.0                                   # singular
    A[5] = np.diag(np.r_[np.ones(f - 1), 1e-8])  # pivot ratio 1e8
    A[8] = 0.0                                   # singular, last
    A = A.astype(np.float32)
    b = rng.standard_normal((n, f)).astype(np.float32)
    eng = core.CoreALS(f, 0.05, 0.25, gram_mode=mode)
    X, flags = eng.solve(torch.as_tensor(A).cuda(), torch.as_tensor(b).cuda())
    Xo, fo, _ = oracle.solve_batch(A.astype(np.float64), b.astype(np.float64), 0 if mode == "asym" else 1)
    flags, X = flags.cpu().numpy(), X.cpu().numpy()
    assert np.array_equal(flags, fo), (flags, fo)
    assert flags[2] & 2 and flags[8] & 2 and flags[5] == 1
    assert np.all(X[2] == 0) and np.all(X[8] == 0)
    ok = [i for i in range(n) if fo[i] == 0]
    assert rel_fro(X[ok], Xo[ok]) <= 1e-4


# -------------------------------------------------------- full runs / e2e
def test_fit_small_rmse_matches_oracle(core, small):
    M0 = synth.init_factor(small.n_m, small.f, 1000)
    for mode, r in (("asym", 0.5), ("full", 1.0)):
        eng = core.CoreALS(small.f, f32(0.1), r, gram_mode=mode)
        Ru = core.DeviceCSR.from_host(small.train_rows)
        Ri = core.DeviceCSR.from_host(small.train_cols)
        test = tuple(torch.as_tensor(a).cuda() for a in (small.test_u, small.test_m, small.test_r))
        U, M, rep = eng.fit(Ru, Ri, torch.as_tensor(M0).cuda(), 10, test=test)
        Uo, Mo = oracle.fit(small.train_rows, small.train_cols, M0, f32(0.1), r, 10, MODES[mode])
        ro = oracle.rmse(small.test_u, small.test_m, small.test_r, Uo, Mo)
        assert abs(rep["test_rmse"] - ro) <= 1e-3 * ro, (mode, rep["test_rmse"], ro)
        # The GPU's own SSE equals the oracle's SSE on the GPU factors.
        sse_o = oracle.sse(small.test_u, small.test_m, small.test_r, U.cpu().numpy(), M.cpu().numpy())
        assert rep["test_rmse"] == pytest.approx(np.sqrt(sse_o / len(small.test_r)), rel=1e-6)


def test_fit_host_equals_device_path(core, small):
    M0 = synth.init_factor(small.n_m, small.f, 1000)
    eng = core.CoreALS(small.f, f32(0.1), 0.5)
    U1, M1, rep1 = eng.fit_host(small.train_rows, small.train_cols, M0, 3,
                                test=(small.test_u, small.test_m, small.test_r))
    U2, M2, rep2 = eng.fit(core.DeviceCSR.from_host(small.train_rows), core.DeviceCSR.from_host(small.train_cols),
                           torch.as_tensor(M0).cuda(), 3,
                           test=tuple(torch.as_tensor(a).cuda() for a in (small.test_u, small.test_m, small.test_r)))
    assert np.array_equal(U1, U2.cpu().numpy()) and np.array_equal(M1, M2.cpu().numpy())
    assert rep1["test_rmse"] == rep2["test_rmse"]


def test_fit_host_pipelined_inputs(core, small):
    # als_fit_host copies and validates the item side on its copy stream under
    # the first user half-sweep: 0, 1 and 2 sweeps, repeated calls on the same
    # structure (plans kept), and an invalid item side (rejected; the handle
    # stays usable) all match the device-buffer path.
    M0 = synth.init_factor(small.n_m, small.f, 1000)
    test = (small.test_u, small.test_m, small.test_r)
    eng = core.CoreALS(small.f, f32(0.1), 0.5)
    Ru, Ri = core.DeviceCSR.from_host(small.train_rows), core.DeviceCSR.from_host(small.train_cols)
    dtest = tuple(torch.as_tensor(a).cuda() for a in test)
    for sweeps in (0, 1, 2, 2):
        U1, M1, rep1 = eng.fit_host(small.train_rows, small.train_cols, M0, sweeps, test=test)
        U2, M2, rep2 = eng.fit(Ru, Ri, torch.as_tensor(M0).cuda(), sweeps, test=dtest)
        assert np.array_equal(M1, M2.cpu().numpy()), sweeps
        assert rep1["sweeps_done"] == sweeps
        if sweeps:  # (with none, U is the caller's initial buffer on each path)
            assert np.array_equal(U1, U2.cpu().numpy()), sweeps
            assert rep1["test_rmse"] == rep2["test_rmse"]
    bad = small.train_cols
    bad_idx = bad.indices.copy()
    bad_idx[bad.indptr[1]] = small.n_u  # out of range in the second item row
    bad = synth.CSR(bad.n_rows, bad.n_cols, bad.indptr, bad_idx, bad.values)
    with pytest.raises(Exception, match="out of range"):
        eng.fit_host(small.train_rows, bad, M0, 1, test=test)
    U1, M1, _ = eng.fit_host(small.train_rows, small.train_cols, M0, 1, test=test)
    U2, M2, _ = eng.fit(Ru, Ri, torch.as_tensor(M0).cuda(), 1, test=dtest)
    assert np.array_equal(U1, U2.cpu().numpy()) and np.array_equal(M1, M2.cpu().numpy())


def test_deterministic(core, small):
    M0 = torch.as_tensor(synth.init_factor(small.n_m, small.f, 5)).cuda()
    eng = core.CoreALS(small.f, 0.1, 0.5)
    Ru = core.DeviceCSR.from_host(small.train_rows)
    a = eng.half_sweep(Ru, M0).cpu().numpy()
    b = eng.half_sweep(Ru, M0).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("f,prec", [(32, 0), (64, 0), (128, 2)])
def test_split_chain_on_second_stream_is_bit_identical(core, f, prec):
    # Without per-launch profiling the split-row chain runs on the handle's
    # second stream beside the resident rows; with it, everything runs on one
    # stream in order. Both write disjoint rows: the results must agree bit
    # for bit (n_f = 32 on CUDA cores; 64 and 128 on the tensor cores).
    csr, Y = rows_problem(LENGTHS + [5000], 6000, f, seed=31)
    eng = core.CoreALS(f, 0.05, 0.25, precision=prec)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    flags_a = torch.zeros(csr.n_rows, dtype=torch.int32, device="cuda")
    flags_b = torch.zeros(csr.n_rows, dtype=torch.int32, device="cuda")
    Xa = eng.half_sweep(R, Yd, flags=flags_a).cpu().numpy()
    eng.profile(True)
    Xb = eng.half_sweep(R, Yd, flags=flags_b).cpu().numpy()
    eng.profile(False)
    assert np.array_equal(Xa, Xb)
    assert np.array_equal(flags_a.cpu().numpy(), flags_b.cpu().numpy())


# ------------------------------------------------------------ bad inputs
def test_bad_structure_is_rejected(core):
    from paper_2509_18024_gb300.binding import AlsError
    csr, Y = rows_problem([3, 4], 10, 8, seed=1)
    eng = core.CoreALS(8, 0.1, 0.5)
    bad = synth.CSR(csr.n_rows, csr.n_cols, csr.indptr, csr.indices.copy(), csr.values)
    bad.indices[0], bad.indices[1] = bad.indices[1], bad.indices[0]
    with pytest.raises(AlsError) as e:
        eng.half_sweep(core.DeviceCSR.from_host(bad), torch.as_tensor(Y).cuda())
    assert e.value.status == -2
    nanv = synth.CSR(csr.n_rows, csr.n_cols, csr.indptr, csr.indices, csr.values.copy())
    nanv.values[2] = np.nan
    with pytest.raises(AlsError) as e:
        eng.half_sweep(core.DeviceCSR.from_host(nanv), torch.as_tensor(Y).cuda())
    assert e.value.status == -3
    oob = synth.CSR(csr.n_rows, csr.n_cols, csr.indptr, csr.indices.copy(), csr.values)
    oob.indices[-1] = 10
    with pytest.raises(AlsError) as e:
        eng.half_sweep(core.DeviceCSR.from_host(oob), torch.as_tensor(Y).cuda())
    assert e.value.status == -2


# -------------------------------------------- the benchmark's full workload
@pytest.fixture(scope="module")
def zipf():
    return synth.make_workload("zipf_100k")


@pytest.mark.parametrize("side", ["users", "items"])
def test_full_size_sampled_rows(core, zipf, side):
    """The 100k x 20k, 10M-entry, n_f = 32 workload in the benchmark's launch
    configuration: all rows on the GPU, a sample (incl. the longest rows)
    compared with the oracle row by row, masks bit-exact on the sample."""
    f, lam, r = 32, f32(0.05), 0.25
    M0 = synth.init_factor(zipf.n_m, f, 1000)
    if side == "users":
        csr, Y = zipf.train_rows, M0
    else:
        # Item side from a seeded user factor (an oracle user sweep over all
        # 100k users would take minutes on the host).
        csr, Y = zipf.train_cols, synth.init_factor(zipf.n_u, f, 2000)
    X, flags, masks, _ = gpu_half(core, csr, Y, f, lam, r)
    L = np.diff(csr.indptr)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([np.argsort(L)[-20:], rng.choice(csr.n_rows, 400, replace=False)]))
    Xo, fo, _ = oracle_half(csr, Y, lam, r, rows=sample)
    err = rel_fro(X[sample], Xo[sample])
    assert err <= HALF_TOL, err
    # Masks of the sampled rows, from a CSR holding only those rows.
    lens = L[sample]
    sub_ptr = np.zeros(len(sample) + 1, np.int64)
    np.cumsum(lens, out=sub_ptr[1:])
    take = np.concatenate([np.arange(csr.indptr[i], csr.indptr[i + 1]) for i in sample])
    mo = oracle.select_half(sub_ptr, csr.indices[take], Y.astype(np.float64), r)
    assert np.array_equal(masks[take], mo)


def test_refilled_buffers_with_invalid_entries_are_reported(core):
    # A cached plan trusts its buffers' identity; refilling them in place with
    # an out-of-range index or a NaN rating is caught by the device-side check
    # that every reuse runs, and the next report returns the error. The
    # clamped gathers keep the results finite meanwhile.
    from paper_2509_18024_gb300 import binding as B
    csr, Y = rows_problem(LENGTHS, 4000, 32, seed=9)
    eng = core.CoreALS(32, 0.05, 0.25)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    X = eng.half_sweep(R, Yd)
    eng.report()
    for field, at, bad, status in (("indices", 40, 4007, -2), ("values", 41, float("nan"), -3),
                                   ("indices", 5500, -3, -2)):
        buf = getattr(R, field)
        keep = buf[at].item()
        buf[at] = bad
        X = eng.half_sweep(R, Yd)
        assert torch.isfinite(X).all() or field == "values"
        with pytest.raises(B.AlsError) as e:
            eng.report()
        assert e.value.status == status, (field, e.value.status)
        buf[at] = keep
        X = eng.half_sweep(R, Yd)
        eng.report()  # clean again
    Xo, _, _ = oracle_half(csr, Y, 0.05, 0.25)
    assert rel_fro(X.cpu().numpy(), Xo) <= HALF_TOL

"""FP64 fallback for flagged rows and one iterative-refinement step.

* Rows whose FP32 pivot ratio exceeds pivot_ratio_max are re-assembled from
  the data and re-solved in FP64: they carry ALS_FLAG_FP64 and match the
  FP64 oracle up to the FP32 rounding of the stored result (same FP32
  inputs, same selection, FP64 arithmetic): 2^-24 per component, bounded
  here by 2e-7 of the row norm.
* One refinement step (residual from the FP32 data, correction solved with
  the same assembled G) shrinks the error of the BF16 / TF32 Gram by at
  least an order of magnitude on the rows it covers (rows with more than 32
  observations; shorter rows are assembled in FP32 anyway).
"""
import numpy as np
import pytest

import oracle
from paper_2509_18024_gb300 import synth
from tests.helpers import rel_fro, rows_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32, TF32, BF16 = 0, 1, 2
FLAG_FP64 = 4


@pytest.fixture(scope="module")
def core():
    from paper_2509_18024_gb300 import core_als
    return core_als


def f32(x):
    return float(np.float32(x))


@pytest.mark.parametrize("f,prec", [(10, FP32), (32, FP32), (64, FP32), (32, BF16)])
def test_fp64_fallback_on_ill_conditioned_rows(core, f, prec):
    # Plain lambda = 0.1 and r = 0.25 leave rows with condition numbers ~1e4.
    if f == 10:
        p = synth.make_workload("small")
        csr, Y = p.train_rows, synth.init_factor(p.n_m, p.f, 1001)
        lam = f32(0.1)
    else:
        csr, Y = rows_problem([8, 12, 20, 25, 40, 60, 200, 1500] * 20, 3000, f, seed=f)
        lam = f32(0.01)
    r = 0.25
    eng = core.CoreALS(f, lam, r, reg_mode="plain", ratio_max=1e3, precision=prec)
    R = core.DeviceCSR.from_host(csr)
    flags = torch.zeros(csr.n_rows, dtype=torch.int32, device="cuda")
    X = eng.half_sweep(R, torch.as_tensor(Y).cuda(), flags=flags).cpu().numpy()
    rep = eng.report()
    flags = flags.cpu().numpy()
    Xo, fo, ratios = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), lam, r,
                                       oracle.GRAM_ASYM, oracle.REG_PLAIN, ratio_max=1e3)
    redo = (flags & FLAG_FP64) != 0
    assert redo.sum() == rep["rows_fp64"] > 0
    # Every row whose FP64 pivot ratio is well above the threshold was redone.
    assert np.all(redo[ratios > 1e4])
    for i in np.nonzero(redo)[0]:
        nx = np.linalg.norm(Xo[i])
        if nx > 0:
            assert np.linalg.norm(X[i] - Xo[i]) <= 2e-7 * nx, (i, ratios[i])


def test_fallback_off_leaves_rows_flagged_only(core):
    p = synth.make_workload("small")
    Y = synth.init_factor(p.n_m, p.f, 1001)
    eng = core.CoreALS(p.f, 0.1, 0.25, reg_mode="plain", ratio_max=1e3, fp64_fallback=False)
    flags = torch.zeros(p.n_u, dtype=torch.int32, device="cuda")
    eng.half_sweep(core.DeviceCSR.from_host(p.train_rows), torch.as_tensor(Y).cuda(), flags=flags)
    flags = flags.cpu().numpy()
    assert np.all((flags & FLAG_FP64) == 0) and np.any(flags & 1)
    assert eng.report()["rows_fp64"] == 0


@pytest.mark.parametrize("f,prec", [(32, BF16), (32, TF32), (64, BF16), (128, TF32)])
def test_refinement_step_shrinks_mixed_precision_error(core, f, prec):
    csr, Y = rows_problem([40, 80, 150, 300, 700, 1500] * 30, 3000, f, seed=2 * f + prec)
    lam, r = f32(0.05), 0.25
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), lam, r)
    errs = []
    for steps in (0, 1, 2):
        eng = core.CoreALS(f, lam, r, precision=prec, refine_steps=steps)
        X = eng.half_sweep(core.DeviceCSR.from_host(csr), torch.as_tensor(Y).cuda()).cpu().numpy()
        errs.append(rel_fro(X, Xo))
    print(f"f={f} prec={prec} error after 0 / 1 / 2 refinement steps: {errs[0]:.3e} / {errs[1]:.3e} / {errs[2]:.3e}")
    assert errs[1] <= errs[0] / 10
    # A second step contracts again until the FP32 solve's own error is reached.
    assert errs[2] <= max(errs[1] / 4, 2e-6)


def test_refinement_keeps_fp32_at_parity(core):
    csr, Y = rows_problem([40, 80, 150, 300, 700, 1500] * 10, 3000, 32, seed=9)
    lam, r = f32(0.05), 0.25
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), lam, r)
    eng = core.CoreALS(32, lam, r, refine_steps=1)
    X = eng.half_sweep(core.DeviceCSR.from_host(csr), torch.as_tensor(Y).cuda()).cpu().numpy()
    assert rel_fro(X, Xo) <= 1e-5


def test_bounded_wait_runs_out_reports_and_handle_stays_usable(core):
    # A wait on a barrier that nothing arrives at gives up after its limit,
    # the device error word records it, the host call returns
    # ALS_ERR_TIMEOUT, and the record is cleared: the handle keeps working.
    from paper_2509_18024_gb300 import binding as B
    csr, Y = rows_problem([0, 5, 40, 300, 2000], 3000, 64, seed=41)
    eng = core.CoreALS(64, 0.05, 0.25)
    with pytest.raises(B.AlsError) as e:
        eng._call(eng.lib.als_wait_selftest, 1_000_000, 0)  # 1 ms of GPU time
    assert e.value.status == -5 and B.STATUS[-5] == "ALS_ERR_TIMEOUT"
    # Cleared: the next report is clean, and a half-sweep (tensor-core Gram
    # at n_f = 64) still matches the oracle.
    R = core.DeviceCSR.from_host(csr)
    X = eng.half_sweep(R, torch.as_tensor(Y).cuda()).cpu().numpy()
    eng.report()
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), f32(0.05), 0.25,
                                 oracle.GRAM_ASYM)
    assert rel_fro(X, Xo) <= 1e-5
    with pytest.raises(B.AlsError):
        eng._call(eng.lib.als_wait_selftest, -1, 0)


def test_fit_without_report_still_returns_a_timeout(core):
    # The record left by a wait that ran out must reach the caller of
    # als_fit even when no report is asked for; the next fit is clean.
    import ctypes
    from paper_2509_18024_gb300 import binding as B
    p = synth.make_workload("small")
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    eng = core.CoreALS(p.f, 0.1, 0.5)
    M = torch.as_tensor(synth.init_factor(p.n_m, p.f, 1000)).cuda()
    U = torch.empty((p.n_u, p.f), device="cuda")
    eng._call(eng.lib.als_wait_selftest, 1_000_000, 1)  # leaves the record
    args = (ctypes.byref(Ru.c_struct()), ctypes.byref(Ri.c_struct()), 2, B.ptr(U), B.ptr(M), 0, None, None, None,
            None)
    with pytest.raises(B.AlsError) as e:
        eng._call(eng.lib.als_fit, *args)
    assert e.value.status == -5
    eng._call(eng.lib.als_fit, *args)

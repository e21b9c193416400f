"""Tensor-core (tcgen05) Gram assembly: widths 32, 64, 128 and the precision
modes, against the FP64 oracle.

* ALS_FP32_TC / ALS_FP32 above 32 features (split TF32: x = hi + lo,
  hi*hi + hi*lo + lo*hi in FP32): same 1e-5 bar as the CUDA-core FP32 path.
* ALS_TF32 / ALS_BF16: inputs rounded to 11 / 8 significant bits. The
  half-sweep error is reported and bounded by c * kappa_typ * u with
  u = 2^-11 (TF32) or 2^-8 (BF16); kappa of the weighted-lambda systems on
  these inputs is below ~20, c = 4 covers the Gram and the solve.
* Masks are independent of the precision and stay bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_2509_18024_gb300 import synth
from tests.helpers import rel_fro, rows_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32, TF32, BF16, FP32_TC = 0, 1, 2, 3
BOUND = {FP32: 1e-5, FP32_TC: 1e-5, TF32: 4 * 20 * 2.0 ** -11, BF16: 4 * 20 * 2.0 ** -8}
MODES = {"asym": oracle.GRAM_ASYM, "sym": oracle.GRAM_SYM, "full": oracle.GRAM_FULL}
# Covers every bucket of widths 64 and 128, split rows included.
LENGTHS = [0, 1, 2, 5, 17, 31, 32, 33, 40, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256, 257, 511, 512, 513,
           700, 1500]


@pytest.fixture(scope="module")
def core():
    from paper_2509_18024_gb300 import core_als
    return core_als


def f32(x):
    return float(np.float32(x))


def run(core, csr, Y, f, lam, r, prec, mode="asym"):
    eng = core.CoreALS(f, lam, r, gram_mode=mode, precision=prec)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    X = eng.half_sweep(R, Yd).cpu().numpy()
    masks = eng.select(R, Yd).cpu().numpy().view(np.uint32)
    return X, masks


@pytest.mark.parametrize("f", [24, 32, 48, 64, 100, 128])
@pytest.mark.parametrize("prec", [FP32, FP32_TC, TF32, BF16])
def test_widths_and_precisions(core, f, prec):
    csr, Y = rows_problem(LENGTHS, 3000, f, seed=f + 7)
    lam, r = f32(0.05), 0.25
    X, masks = run(core, csr, Y, f, lam, r, prec)
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), lam, r)
    mo = oracle.select_half(csr.indptr, csr.indices, Y.astype(np.float64), r)
    assert np.array_equal(masks, mo)
    err = rel_fro(X, Xo)
    print(f"f={f} prec={prec} rel err {err:.3e}")
    assert err <= BOUND[prec], err


@pytest.mark.parametrize("f", [64, 128])
@pytest.mark.parametrize("mode,r", [("sym", 0.5), ("full", 1.0), ("asym", 0.1)])
def test_wide_modes_fp32(core, f, mode, r):
    csr, Y = rows_problem(LENGTHS, 3000, f, seed=3 * f)
    X, _ = run(core, csr, Y, f, f32(0.05), r, FP32, mode)
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), f32(0.05), r,
                                 MODES[mode])
    assert rel_fro(X, Xo) <= 1e-5


def test_wide_ties_masks(core):
    pool = [0.0, -0.0, 0.5, -0.5, 1.0, -1.0, 0.25]
    for f in (64, 128):
        csr, Y = rows_problem(LENGTHS, 3000, f, seed=f, pool=pool)
        for r in (0.1, 0.5):
            _, masks = run(core, csr, Y, f, 0.05, r, TF32)
            mo = oracle.select_half(csr.indptr, csr.indices, Y.astype(np.float64), r)
            assert np.array_equal(masks, mo)


@pytest.mark.parametrize("prec", [TF32, BF16])
def test_mixed_precision_fit_reaches_fp32_rmse(core, prec):
    """Mixed-precision Gram (tensor cores) with the automatic refinement
    steps (one for TF32, two for BF16) reaches the FP32 test RMSE within 1e-3
    relative after the same number of sweeps on the small workload."""
    p = synth.make_workload("small")
    M0 = torch.as_tensor(synth.init_factor(p.n_m, p.f, 1000)).cuda()
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    test = tuple(torch.as_tensor(a).cuda() for a in (p.test_u, p.test_m, p.test_r))
    out = {}
    for pr in (FP32, prec):
        eng = core.CoreALS(p.f, f32(0.1), 0.5, precision=pr)
        _, _, rep = eng.fit(Ru, Ri, M0, 10, test=test)
        out[pr] = rep["test_rmse"]
    assert abs(out[prec] - out[FP32]) <= 1e-3 * out[FP32], out

"""Autotuned row schedules: every candidate keeps parity with the oracle, and
als_autotune picks one, restores M and caches the choice."""
import numpy as np
import pytest

import oracle
from tests.helpers import rel_fro, rows_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LENGTHS = [0, 1, 5, 31, 32, 33, 100, 128, 129, 300, 511, 512, 513, 900, 1024, 1025, 3000]


@pytest.fixture(scope="module")
def core():
    from paper_2509_18024_gb300 import core_als
    return core_als


@pytest.mark.parametrize("split,warp,tc", [(0, 1, 0), (1, 1, 0), (0, 0, 0), (1, 0, 1), (0, 1, 1)])
def test_every_schedule_keeps_parity(core, split, warp, tc):
    csr, Y = rows_problem(LENGTHS * 3, 4000, 32, seed=13)
    lam, r = float(np.float32(0.05)), 0.25
    eng = core.CoreALS(32, lam, r)
    eng.set_tuning(split, warp, tc)
    R = core.DeviceCSR.from_host(csr)
    Yd = torch.as_tensor(Y).cuda()
    X = eng.half_sweep(R, Yd).cpu().numpy()
    masks = eng.select(R, Yd).cpu().numpy().view(np.uint32)
    Xo, _, _ = oracle.half_sweep(csr.indptr, csr.indices, csr.values, Y.astype(np.float64), lam, r)
    mo = oracle.select_half(csr.indptr, csr.indices, Y.astype(np.float64), r)
    assert np.array_equal(masks, mo)
    assert rel_fro(X, Xo) <= 1e-5


def test_autotune_picks_and_caches(core):
    from paper_2509_18024_gb300 import synth
    p = synth.make_workload("small", n_u=3000, n_m=1500, f=32, density=0.03)
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    M = torch.as_tensor(synth.init_factor(p.n_m, 32, 5)).cuda()
    M_in = M.clone()
    U = torch.empty((p.n_u, 32), device="cuda")
    eng = core.CoreALS(32, 0.1, 0.25)
    t = eng.autotune(Ru, Ri, U, M, trials=2)
    assert t["ms_per_sweep"] > 0
    assert torch.equal(M, M_in)
    eng2 = core.CoreALS(32, 0.1, 0.25)
    t2 = eng2.autotune(Ru, Ri, U, M, trials=2)  # cached: same choice, no timing
    assert (t2["split_at_middle"], t2["warp_rows"], t2["tc_gram"]) == (t["split_at_middle"], t["warp_rows"],
                                                                       t["tc_gram"])
    # A fit with the tuned schedule still reaches the untuned test RMSE.
    test = tuple(torch.as_tensor(a).cuda() for a in (p.test_u, p.test_m, p.test_r))
    _, _, rep_t = eng.fit(Ru, Ri, M_in, 5, test=test)
    _, _, rep_0 = core.CoreALS(32, 0.1, 0.25).fit(Ru, Ri, M_in, 5, test=test)
    assert abs(rep_t["test_rmse"] - rep_0["test_rmse"]) <= 1e-3 * rep_0["test_rmse"]

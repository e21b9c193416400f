"""Batched independent problems (als_batch_*) and graph-replayed fits.

Problems of one width are concatenated block-diagonally and share launches;
rows never interact, so every problem must come out bit-identical to the same
problem fitted alone. als_fit replays a captured CUDA graph after its first
sweep; that must also be bit-identical to direct sweeps.
"""
import numpy as np
import pytest

from paper_2509_18024_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def core():
    from paper_2509_18024_gb300 import core_als
    return core_als


def small_problem(seed, n_u, n_m, f, density):
    p = synth.uniform_lowrank(n_u, n_m, f, density, 0.1, seed)
    return p


@pytest.mark.parametrize("prec", [0, 2])
def test_batch_equals_individual_fits(core, prec):
    specs = [(1, 300, 200, 8, 0.08), (2, 500, 300, 16, 0.05), (3, 400, 250, 8, 0.1), (4, 800, 400, 32, 0.04),
             (5, 300, 300, 10, 0.2), (6, 600, 200, 64, 0.1), (7, 1200, 2500, 32, 0.03)]
    if prec == 2:
        specs = [s for s in specs if s[3] >= 32 or s[3] == 16]
    problems, refs = [], []
    for seed, n_u, n_m, f, d in specs:
        p = small_problem(seed, n_u, n_m, f, d)
        Ru = core.DeviceCSR.from_host(p.train_rows)
        Ri = core.DeviceCSR.from_host(p.train_cols)
        M0 = torch.as_tensor(synth.init_factor(n_m, f, 100 + seed)).cuda()
        U = torch.zeros((n_u, f), device="cuda")
        problems.append((Ru, Ri, f, U, M0.clone()))
        eng = core.CoreALS(f, 0.1, 0.5, precision=prec)
        Ui, Mi, _ = eng.fit(Ru, Ri, M0, 4)
        refs.append((Ui.cpu().numpy(), Mi.cpu().numpy()))
    batch = core.CoreBatch(problems, 0.1, 0.5, precision=prec)
    batch.fit(4).synchronize()
    assert batch.launches_per_sweep > 0
    for (Ru, Ri, f, U, M), (Ur, Mr) in zip(problems, refs):
        assert np.array_equal(U.cpu().numpy(), Ur)
        assert np.array_equal(M.cpu().numpy(), Mr)
    # A second fit restarts from the M each problem holds now.
    batch.fit(1).synchronize()
    batch.close()


def test_graph_replayed_fit_equals_direct_sweeps(core):
    p = synth.make_workload("small")
    Ru = core.DeviceCSR.from_host(p.train_rows)
    Ri = core.DeviceCSR.from_host(p.train_cols)
    M0 = torch.as_tensor(synth.init_factor(p.n_m, p.f, 1000)).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        eng = core.CoreALS(p.f, 0.1, 0.5)
        U1, M1, _ = eng.fit(Ru, Ri, M0, 6)
        M2 = M0.clone()
        U2 = torch.empty_like(U1)
        for _ in range(6):
            eng.sweep(Ru, Ri, U2, M2)
    s.synchronize()
    assert np.array_equal(U1.cpu().numpy(), U2.cpu().numpy())
    assert np.array_equal(M1.cpu().numpy(), M2.cpu().numpy())


def test_batch_matches_the_oracle(core):
    """Every problem of a mixed batch (widths 8, 16, 32 and 64, one problem
    with rows long enough to take the split path) against the FP64 oracle:
    each half-sweep of the first sweep from identical inputs within 1e-5
    relative Frobenius error, the masks of the block-diagonal structure
    bit-exact, and the test RMSE after 10 sweeps within 1e-3 relative."""
    import oracle
    from tests.helpers import rel_fro
    lam, r = float(np.float32(0.1)), 0.5
    specs = [(11, 400, 300, 8, 0.06), (12, 500, 350, 12, 0.05), (13, 700, 400, 32, 0.04), (14, 300, 500, 50, 0.1),
             (15, 1400, 1300, 32, 0.85), (16, 600, 700, 64, 0.9)]
    probs, problems = [], []
    for seed, n_u, n_m, f, d in specs:
        p = small_problem(seed, n_u, n_m, f, d)
        M0 = synth.init_factor(n_m, f, 500 + seed)
        Ru = core.DeviceCSR.from_host(p.train_rows)
        Ri = core.DeviceCSR.from_host(p.train_cols)
        problems.append((Ru, Ri, f, torch.zeros((n_u, f), device="cuda"), torch.as_tensor(M0).cuda()))
        probs.append((p, M0))
    assert max(np.diff(probs[4][0].train_rows.indptr)) > 1024  # split rows at widths <= 32
    assert max(np.diff(probs[5][0].train_rows.indptr)) > 512   # split rows at width 64
    batch = core.CoreBatch(problems, lam, r)
    batch.fit(1).synchronize()
    for q, ((p, M0), (Ru, Ri, f, U, M)) in enumerate(zip(probs, problems)):
        Ug, Mg = U.cpu().numpy(), M.cpu().numpy()
        Uo, _, _ = oracle.half_sweep(p.train_rows.indptr, p.train_rows.indices, p.train_rows.values,
                                     M0.astype(np.float64), lam, r)
        assert rel_fro(Ug, Uo) <= 1e-5, (q, rel_fro(Ug, Uo))
        Mo, _, _ = oracle.half_sweep(p.train_cols.indptr, p.train_cols.indices, p.train_cols.values,
                                     Ug.astype(np.float64), lam, r)
        assert rel_fro(Mg, Mo) <= 1e-5, (q, rel_fro(Mg, Mo))
        mu = batch.select(q, 0, torch.as_tensor(M0).cuda()).cpu().numpy().view(np.uint32)
        assert np.array_equal(mu, oracle.select_half(p.train_rows.indptr, p.train_rows.indices,
                                                     M0.astype(np.float64), r)), q
        mi = batch.select(q, 1, U).cpu().numpy().view(np.uint32)
        assert np.array_equal(mi, oracle.select_half(p.train_cols.indptr, p.train_cols.indices,
                                                     Ug.astype(np.float64), r)), q
    # Ten sweeps from M^(0) again (fit reads each problem's M at its start).
    for (p, M0), prob in zip(probs, problems):
        prob[4].copy_(torch.as_tensor(M0).cuda())
    batch.fit(10).synchronize()
    for q, ((p, M0), (Ru, Ri, f, U, M)) in enumerate(zip(probs, problems)):
        Uo, Mo = oracle.fit(p.train_rows, p.train_cols, M0, lam, r, 10)
        ro = oracle.rmse(p.test_u, p.test_m, p.test_r, Uo, Mo)
        rg = oracle.rmse(p.test_u, p.test_m, p.test_r, U.cpu().numpy(), M.cpu().numpy())
        assert abs(rg - ro) <= 1e-3 * ro, (q, rg, ro)
    batch.close()


def test_batch_refuses_the_fast_variant(core):
    from paper_2509_18024_gb300 import binding as B
    p = small_problem(1, 100, 80, 8, 0.1)
    prob = (core.DeviceCSR.from_host(p.train_rows), core.DeviceCSR.from_host(p.train_cols), 8,
            torch.zeros((100, 8), device="cuda"), torch.zeros((80, 8), device="cuda"))
    with pytest.raises(B.AlsError) as e:
        core.CoreBatch([prob], 0.1, 0.5, sketch="factor")
    assert e.value.status == -8

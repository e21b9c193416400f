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

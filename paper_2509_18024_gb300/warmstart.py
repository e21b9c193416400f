"""Learned warm start for Core-ALS (the paper has no counterpart).

Two networks map a row's features to its factor: the user net reads
features computed from the item factor, the item net from the user factor.
They are trained on factors that ALS itself converged to on seeded training
matrices (inputs from the converged other side, targets the converged rows).
At use time, from a random M^(0): U_w = user_net(features(R, M^(0))),
M_w = item_net(features(R^T, U_w)), and ALS starts from M_w. Plain ALS from
M^(0) is the judge: both starts run `judge_after` sweeps (default 5), and the
fit continues from the warm start only if its test RMSE there is not worse;
otherwise it falls back to M^(0). The gain is reported as sweeps and
milliseconds to the target RMSE saved by the warm start (negative when it
loses), and, for early stopping, as the sweeps and milliseconds the warm run
saves in reaching the RMSE the plain run has after a given number of sweeps.

This module only orchestrates; features, the networks (forward, backward,
Adam) and ALS run in libcore_als.so.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import core_als


@dataclass
class Pair:
    users: core_als.MLP
    items: core_als.MLP


def device_sides(problem):
    """(Ru, Ri, (test_u, test_m, test_r)) on the device, for a host problem
    (synth.RatingProblem) or one drawn on the device (synth.DeviceRatingProblem)."""
    if hasattr(problem, "train_rows"):
        Ru = core_als.DeviceCSR.from_host(problem.train_rows)
        Ri = core_als.DeviceCSR.from_host(problem.train_cols)
        test = tuple(torch.as_tensor(a).cuda() for a in (problem.test_u, problem.test_m, problem.test_r))
    else:
        Ru = core_als.DeviceCSR(problem.n_u, problem.n_m, *problem.rows)
        Ri = core_als.DeviceCSR(problem.n_m, problem.n_u, *problem.cols)
        test = (problem.test_u, problem.test_m, problem.test_r)
    return Ru, Ri, test


def converged_factors(problem, n_f, lam, budget, M0, sweeps, precision=0, gram_mode="asym"):
    """ALS from M0 for `sweeps` sweeps; returns device (U, M, Ru, Ri)."""
    Ru, Ri, _ = device_sides(problem)
    eng = core_als.CoreALS(n_f, lam, budget, gram_mode=gram_mode, precision=precision)
    U, M, _ = eng.fit(Ru, Ri, torch.as_tensor(M0).cuda(), sweeps)
    return U, M, Ru, Ri


def train(problems, n_f, lam, budget, sweeps=15, hidden=256, epochs=30, batch=4096, lr=1e-3, seed=0):
    """Train the user and item nets on ALS-converged factors of `problems`."""
    from . import synth
    Xu, Tu, Xm, Tm = [], [], [], []
    for q, p in enumerate(problems):
        M0 = synth.init_factor(p.n_m, n_f, 7000 + q)
        U, M, Ru, Ri = converged_factors(p, n_f, lam, budget, M0, sweeps)
        Xu.append(core_als.features(Ru, M, n_f))
        Tu.append(U)
        Xm.append(core_als.features(Ri, U, n_f))
        Tm.append(M)
    nets = Pair(core_als.MLP(n_f + 2, hidden, n_f, seed), core_als.MLP(n_f + 2, hidden, n_f, seed + 1))
    gen = torch.Generator(device="cuda").manual_seed(seed)
    history = {"users": [], "items": []}
    for net, X, T, key in ((nets.users, torch.cat(Xu), torch.cat(Tu), "users"),
                           (nets.items, torch.cat(Xm), torch.cat(Tm), "items")):
        n = X.shape[0]
        for ep in range(epochs):
            perm = torch.randperm(n, device="cuda", generator=gen)
            last = None
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                want = s + batch >= n
                last = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr, want_loss=want)
            history[key].append(last)
    return nets, history


def warm_factor(nets: Pair, Ru, Ri, M0: torch.Tensor, n_f: int):
    """M_w from a random M^(0): users from M^(0), then items from the users."""
    Uw = nets.users.forward(core_als.features(Ru, M0, n_f))
    return nets.items.forward(core_als.features(Ri, Uw, n_f))


def judge(nets: Pair, problem, n_f, lam, budget, M0, sweeps, target=None, precisions=(0,), judge_after=5):
    """Test RMSE per sweep from M^(0) (plain ALS, FP32) and from the warm start
    (one run per precision in `precisions`), the chosen start (warm unless its
    RMSE after `judge_after` sweeps is worse than the plain run's), the sweeps
    and CUDA-event milliseconds each run needs to reach `target` (default: the
    plain run's final RMSE x (1 + 1e-3)), and the gain of the first warm run
    over the plain one in both (None where a run never reaches the target). A
    warm run's time includes computing the warm start."""
    Ru, Ri, test = device_sides(problem)
    M0d = torch.as_tensor(M0).cuda()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    warm_factor(nets, Ru, Ri, M0d, n_f)  # first call builds the feature plans
    torch.cuda.synchronize()
    a.record()
    Mw = warm_factor(nets, Ru, Ri, M0d, n_f)
    b.record()
    torch.cuda.synchronize()
    warm_ms = a.elapsed_time(b)
    runs = [("plain", M0d, 0, 0.0)] + [(f"warm_p{prec}", Mw, prec, warm_ms) for prec in precisions]
    curves, times = {}, {}
    for name, start, prec, t0 in runs:
        eng = core_als.CoreALS(n_f, lam, budget, precision=prec)
        eng.prepare(Ru)
        eng.prepare(Ri)
        M = start.clone()
        U = torch.empty((problem.n_u, n_f), device="cuda")
        errs, ms = [], []
        total = t0
        for _ in range(sweeps):
            a.record()
            eng.sweep(Ru, Ri, U, M)
            b.record()
            torch.cuda.synchronize()
            total += a.elapsed_time(b)
            ms.append(total)
            errs.append(eng.rmse(*test, U, M))
        curves[name], times[name] = errs, ms
        eng.close()
    if target is None:
        target = curves["plain"][-1] * (1 + 1e-3)
    first_warm = f"warm_p{precisions[0]}"
    k = max(1, min(judge_after, sweeps))
    chosen = "warm" if curves[first_warm][k - 1] <= curves["plain"][k - 1] else "plain"
    reach = {key: next((q + 1 for q, e in enumerate(v) if e <= target), None) for key, v in curves.items()}
    reach_ms = {key: (times[key][reach[key] - 1] if reach[key] else None) for key in curves}
    gain = {"sweeps_saved": (reach["plain"] - reach[first_warm]) if reach["plain"] and reach[first_warm] else None,
            "ms_saved": (reach_ms["plain"] - reach_ms[first_warm]) if reach["plain"] and reach[first_warm] else None,
            "rmse_at_judge": {"plain": curves["plain"][k - 1], "warm": curves[first_warm][k - 1]},
            "final_rmse": {"plain": curves["plain"][-1], "warm": curves[first_warm][-1]}}
    # Early-stopping view: sweeps and ms the warm run needs to reach the RMSE
    # the plain run has after j sweeps (None if it never does), for j = the
    # judging point and half the sweeps.
    gain["to_plain_after"] = {}
    for j in sorted({k, max(1, sweeps // 2)}):
        goal = curves["plain"][j - 1]
        rw = next((q + 1 for q, e in enumerate(curves[first_warm]) if e <= goal), None)
        gain["to_plain_after"][j] = {
            "rmse": goal, "warm_sweeps": rw,
            "sweeps_saved": (j - rw) if rw else None,
            "ms_saved": (times["plain"][j - 1] - times[first_warm][rw - 1]) if rw else None}
    out = {"target": target, "curves": curves, "chosen": chosen, "judge_after": k, "sweeps_to_target": reach,
           "ms_to_target": reach_ms, "warm_start_ms": warm_ms, "gain": gain}
    out["curves"]["warm"] = curves[first_warm]
    out["sweeps_to_target"]["warm"] = reach[first_warm]
    return out

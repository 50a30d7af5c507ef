"""The checkpointed adjoint of a named workload at a long horizon: one sweep with the
adjoint-energy series E_vhat^n and the per-step sigma_1 statistics (section "Results":
the adjoint energy of the vane LES grows by tens of orders of magnitude over long
horizons, which is what the sigma_1-scaled viscosity of section "Energy analysis"
counters).  Reports the wall time, the binomial checkpointing's replay count (measured
from the plan against the repetition number the slots predict), the growth of E_vhat in
e-folds and the sigma_1 range, and optionally writes the series.

    python -m paper_1511_06959_gb300.horizon_study --workload box512 --nsteps 20000 \
        --lambda-tilde 0 --out series_box512.npz

Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import api
from . import config as C


def predicted_repetitions(slots: int, nsteps: int) -> int:
    """The smallest r with C(slots + r, slots) >= nsteps (binomial checkpointing)."""
    r = 0
    while math.comb(slots + r, slots) < nsteps:
        r += 1
    return r


def run(workload: str, nsteps: int, lam_tilde: float, precision: int) -> tuple:
    wl = C.WORKLOADS[workload]
    w0 = np.ascontiguousarray(wl.initial_state())
    S = api.Solver(wl.nx, wl.ny, wl.nz, wl.dx, gamma=wl.gamma, mu=wl.mu, Pr=wl.Pr, dt=0.0,
                   precision=precision, plane_i=wl.plane_i, pt_in=wl.pt_in, batch=wl.batch)
    w = torch.from_numpy(w0).cuda()
    m = torch.empty(1, dtype=torch.float64, device="cuda")
    S.max_wave_speed(w, m)
    dt = C.cfl_dt(wl, m.item())
    S.set_dt(dt)
    N = nsteps or wl.nsteps
    sched = C.SCHEDULES[wl.schedule]
    param = wl.param if wl.schedule != "revolve" or wl.param else C.revolve_slots(wl, w0.nbytes)
    _, slots_used, advances = api.plan(N, sched, param)
    opts = S.run_opts(N, sched, param, lam_tilde * wl.dx[0] ** 2, 0.0, True, True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(wl.batch, dtype=torch.float64, device="cuda")
    lam0 = torch.empty_like(w)
    E = torch.zeros((N + 1, wl.batch), dtype=torch.float64, device="cuda")
    sig = torch.zeros((N, wl.batch, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.adjoint_run(w, opts, arena, J, lam0, energy=E, sigma_stats=sig)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    Eh = E.cpu().numpy()[:, 0]
    sh = sig.cpu().numpy()[:, 0, :]
    finite = np.isfinite(Eh) & (Eh > 0)
    # growth as the adjoint runs backward: ln E at step 0 over ln E at the last step, and
    # the normalised fit of the library's estimator (accumulation of N - m + 1 sources)
    growth = float(np.log(Eh[0] / Eh[N])) if finite[0] and finite[N] else float("inf")
    efolds = api.energy_efolds(E.cpu().numpy(), N, wl.batch)
    res = {
        "workload": workload, "cells": wl.cells * wl.batch, "nsteps": N, "dt": dt,
        "precision": "fp64" if precision == api.NS_FP64 else "mixed", "lambda_tilde": lam_tilde,
        "schedule": wl.schedule, "param": param, "arena_gb": arena.numel() / 1e9,
        "slots_used": slots_used, "advances": advances, "replays_per_step": advances / N,
        "predicted_repetitions": predicted_repetitions(param, N) if wl.schedule == "revolve" else None,
        "seconds": seconds, "adjoint_cell_steps_per_s": wl.cells * wl.batch * N / seconds,
        "J_bar": float(J[0].item()), "E_first": float(Eh[N]), "E_last": float(Eh[0]),
        "E_max": float(np.max(Eh[finite])) if finite.any() else None,
        "ln_E0_over_EN": growth, "efolds_normalised_fit": efolds,
        "sigma1_max_range": [float(sh[:, 0].min()), float(sh[:, 0].max())],
        "sigma1_mean_range": [float(sh[:, 1].min()), float(sh[:, 1].max())],
        "sticky_error": S.last_error(),
    }
    return res, Eh, sh


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="box512")
    ap.add_argument("--nsteps", type=int, default=20000)
    ap.add_argument("--lambda-tilde", type=float, default=0.0)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--out", default=None, help="write E_vhat and sigma_1 series (.npz)")
    a = ap.parse_args(argv)
    res, Eh, sh = run(a.workload, a.nsteps, a.lambda_tilde, api.NS_FP64 if a.fp64 else api.NS_MIXED)
    print(json.dumps(res))
    if a.out:
        np.savez(a.out, E=Eh, sigma_max=sh[:, 0], sigma_mean=sh[:, 1], summary=json.dumps(res))


if __name__ == "__main__":
    main()

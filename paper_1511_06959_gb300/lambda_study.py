"""Choice of the viscosity scaling factor on a named workload: the stabilised sweep once
per candidate lambda_tilde (nu = lambda_tilde dx^2 sigma_1), the adjoint-energy growth
of each run, the change of the source sensitivity between consecutive runs and the
chosen factor, all from ns_estimate_lambda.

    python -m paper_1511_06959_gb300.lambda_study --workload box128 --out lambda_box128.json

Prints (and optionally writes) one JSON object with the candidates, the reports, the
choice and the wall time of the whole scan.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import api
from . import config as C

DEFAULT_TILDES = (0.0, 0.0125, 0.025, 0.05, 0.1, 0.2, 0.4)


def run(workload: str, tildes, precision: int, efold_tol: float, rel_tol: float, nsteps: int = 0) -> dict:
    wl = C.WORKLOADS[workload]
    w0 = np.ascontiguousarray(wl.initial_state())
    S = api.Solver(wl.nx, wl.ny, wl.nz, wl.dx, gamma=wl.gamma, mu=wl.mu, Pr=wl.Pr, dt=0.0,
                   precision=precision, plane_i=wl.plane_i, pt_in=wl.pt_in, batch=wl.batch)
    w = torch.from_numpy(w0).cuda()
    m = torch.empty(1, dtype=torch.float64, device="cuda")
    S.max_wave_speed(w, m)
    S.set_dt(C.cfl_dt(wl, m.item()))
    N = nsteps or wl.nsteps
    param = wl.param if wl.schedule != "revolve" or wl.param else C.revolve_slots(wl, w0.nbytes)
    opts = S.run_opts(N, C.SCHEDULES[wl.schedule], param)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    work = torch.empty(S.estimate_work_bytes(opts), dtype=torch.uint8, device="cuda")
    lambdas = [t * wl.dx[0] ** 2 for t in tildes]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    chosen, ef, ch = S.estimate_lambda(w, opts, lambdas, arena, work, efold_tol=efold_tol, rel_tol=rel_tol)
    seconds = time.perf_counter() - t0
    return {
        "workload": workload, "nsteps": N, "precision": "fp64" if precision == api.NS_FP64 else "mixed",
        "lambda_tilde": list(tildes), "efolds": ef, "change": ch, "efold_tol": efold_tol, "rel_tol": rel_tol,
        "chosen_index": chosen, "chosen_lambda_tilde": tildes[chosen] if chosen >= 0 else None,
        "seconds": seconds, "sticky_error": S.last_error(),
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="box128")
    ap.add_argument("--tildes", default=",".join(str(t) for t in DEFAULT_TILDES))
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--nsteps", type=int, default=0)
    ap.add_argument("--efold-tol", type=float, default=1.0)
    ap.add_argument("--rel-tol", type=float, default=0.1)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    tildes = tuple(float(t) for t in a.tildes.split(","))
    res = run(a.workload, tildes, api.NS_FP64 if a.fp64 else api.NS_MIXED, a.efold_tol, a.rel_tol, a.nsteps)
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()

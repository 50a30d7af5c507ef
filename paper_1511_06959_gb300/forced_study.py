"""The adjoint of a statistically stationary turbulent box: a periodic box driven by a
time-constant Kolmogorov shear force on the x-momentum equation (synth.kolmogorov_forcing)
is spun up from the laminar shear profile the force sustains, with noise, until the
profile's instability has grown into turbulence; then the
checkpointed adjoint of the pressure loss runs over a horizon from that state, and its
adjoint energy growth (section "Results": the adjoint of a turbulent flow grows
exponentially; section "Energy analysis": the sigma_1-scaled viscosity counters it) is
fitted, and optionally the viscosity scaling factor is chosen over candidates
(ns_estimate_lambda).

The forcing amplitude follows from the laminar Kolmogorov profile it would sustain:
u_1 = U0 sin(2 pi y / L_y) with mu (2 pi / L_y)^2 U0 = amp, at the forcing Reynolds number
Re_f = rho U0 L_y / mu.

    python -m paper_1511_06959_gb300.forced_study --spinup 6000 --nsteps 2000 \
        --lambdas 0,0.05,0.1,0.2,0.4,0.8 --out forced128.json

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
from . import closure
from . import synth


def separation(S, w, s, nsteps, eps=1e-9, seed=17):
    """Growth of a small perturbation of w along the forced trajectory: two primal runs
    from w and w + eps r (r seeded, unit rms per component), the rms difference recorded
    every nsteps // 20 steps.  A chaotic flow separates exponentially at its leading
    Lyapunov exponent, which bounds the adjoint's growth rate from below."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    r = torch.randn(w.shape, generator=g, dtype=torch.float64).to(w.device)
    a, a2 = w.clone(), w + eps * r
    b, b2 = torch.empty_like(a), torch.empty_like(a)
    d0 = float((a2 - a).pow(2).mean().sqrt())
    out = []
    every = max(1, nsteps // 20)
    for n in range(nsteps):
        S.primal_step(a, b, s)
        S.primal_step(a2, b2, s)
        a, b = b, a
        a2, b2 = b2, a2
        if (n + 1) % every == 0:
            out.append((n + 1, float((a2 - a).pow(2).mean().sqrt()) / d0))
    return out


def jbar(S, w, s, nsteps):
    """J-bar = (1/N) sum_{n=1..N} J(w^n) along the forced trajectory from w (the
    time average the sweeps differentiate), stepped without checkpoints."""
    J = torch.zeros(1, dtype=torch.float64, device=w.device)
    a, b = w.clone(), torch.empty_like(w)
    for _ in range(nsteps):
        S.primal_step(a, b, s)
        a, b = b, a
        S.objective(a, J, 1.0 / nsteps)
    return float(J.item())


def finite_differences(S, w, s, nsteps, fd_eps):
    """Central differences of J-bar in the forcing amplitude, s(theta) = (1 + theta) s,
    one per relative step in fd_eps, over a horizon of nsteps; their mean is the
    reference sensitivity (section "Results" compares the stabilised adjoint with finite
    differences of the long-time average, Table 2)."""
    rows = []
    for e in fd_eps:
        Jp = jbar(S, w, (1.0 + e) * s, nsteps)
        Jm = jbar(S, w, (1.0 - e) * s, nsteps)
        rows.append({"rel_step": e, "J_plus": Jp, "J_minus": Jm, "dJ_dtheta": (Jp - Jm) / (2.0 * e)})
    return {"nsteps": nsteps, "rows": rows, "mean_dJ_dtheta": float(np.mean([r["dJ_dtheta"] for r in rows]))}


def sensitivity_scan(S, w, s, nsteps, stride, lambdas, dx0):
    """Sensitivity of J-bar to the forcing amplitude, s(theta) = (1 + theta) s at theta = 0,
    as section "Results" compares it (Table 2): dJ-bar/dtheta = <s-bar, s> from the
    stabilised adjoint for each viscosity factor lambda = lambda-tilde dx^2, with its
    adjoint energy growth."""
    dev = w.device
    J = torch.empty(1, dtype=torch.float64, device=dev)
    lam0 = torch.empty_like(w)
    sb = torch.empty_like(w)
    adj = []
    for t in lambdas:
        opts = S.run_opts(nsteps, api.NS_CKPT_STRIDE, stride, t * dx0 ** 2, 0.0, True)
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device=dev)
        E = torch.zeros((nsteps + 1, 1), dtype=torch.float64, device=dev)
        S.adjoint_run(w, opts, arena, J, lam0, s=s, sbar=sb, energy=E)
        adj.append({"lambda_tilde": t, "dJ_dtheta": float((sb * s).sum()),
                    "efolds": api.energy_efolds(E.cpu().numpy(), nsteps, 1)[0], "sticky_error": S.last_error()})
        del arena
    J0 = float(J.item())
    return {"J_bar": J0, "adjoint": adj}


def closure_judge(S, S64, w, s, nsteps, stride, dx0, rule_tildes, kappas, g_ref, label_starts=(0, 2000, 4000),
                  label_steps=100, label_every=5, train_steps=4000, batch=8192, lr=2e-3, cap=False):
    """The learned closure against the sigma_1 rule on the forced box, with finite
    differences of J-bar (g_ref) as the reference (the unstabilised adjoint grows here, so
    it is no reference).  Labels come from short-horizon FP64 adjoints (S64) started at states
    label_starts steps along the forced trajectory from w; the network is trained by the
    library's BF16 kernels; each closure setting is one stabilised sweep over nsteps
    (S, mixed precision), giving dJ-bar/dtheta for s(theta) = (1 + theta) s and the
    adjoint energy E_vhat(w^0, lam^0).  The errors of both closures are compared at the
    energy of the rule's middle setting (log-linear interpolation in the energy).  cap:
    both closures' coefficients held at the explicit stability limit
    (ns_set_viscosity_cap) instead of dropping the settings that exceed it."""
    dev = w.device
    t0 = time.perf_counter()
    feats, targets = [], []
    a, b = w.clone(), torch.empty_like(w)
    done = 0
    for st in label_starts:
        for _ in range(st - done):
            S.primal_step(a, b, s)
            a, b = b, a
        done = st
        smp = closure.generate_samples(S64, a.clone(), label_steps, every=label_every, s=s)
        feats.append(smp.feat)
        targets.append(smp.target)
    feat = torch.cat(feats).contiguous()
    target = torch.cat(targets).contiguous()
    del feats, targets
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = closure.Network(S, closure.init_params(3, out_bias=0.5))
    t0 = time.perf_counter()
    losses = net.train(feat, target, steps=train_steps, batch=batch, lr=lr, seed=2)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    nsamp = int(target.numel())
    del feat, target

    J = torch.empty(1, dtype=torch.float64, device=dev)
    lam0 = torch.empty_like(w)
    sb = torch.empty_like(w)

    def sens(coef, mlp):
        opts = S.run_opts(nsteps, api.NS_CKPT_STRIDE, stride, coef, 0.0, True, False, mlp)
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device=dev)
        E = torch.zeros((nsteps + 1, 1), dtype=torch.float64, device=dev)
        S.adjoint_run(w, opts, arena, J, lam0, s=s, sbar=sb, energy=E)
        return float((sb * s).sum()), float(E[0, 0].item()), S.last_error()

    t0 = time.perf_counter()
    g0, E0, _ = sens(0.0, None)
    S.set_viscosity_cap(cap)

    def sweep(coefs, mlp):
        rows, dropped = [], []
        for cval in coefs:
            g, E, err = sens(cval, mlp)
            if err != 0 or not math.isfinite(g):
                dropped.append(cval)
                continue
            rows.append((cval, g, abs(g - g_ref) / abs(g_ref), E))
        return rows, dropped

    rule, rule_dropped = sweep([t * dx0 ** 2 for t in rule_tildes], None)
    learned, learned_dropped = sweep(list(kappas), net.blob)
    S.set_viscosity_cap(False)
    t_judge = time.perf_counter() - t0
    out = {"samples": nsamp, "cap": bool(cap), "train_loss_first": float(losses[:50].mean()),
           "train_loss_last": float(losses[-50:].mean()),
           "seconds": {"generate": t_gen, "train": t_train, "judge": t_judge},
           "reference_dJ_dtheta": g_ref,
           "unstabilised": {"dJ_dtheta": g0, "E0": E0, "rel_err": abs(g0 - g_ref) / abs(g_ref)},
           "rule": rule, "learned": learned, "rule_dropped_unstable": rule_dropped,
           "learned_dropped_unstable": learned_dropped}
    if len(rule) >= 2 and len(learned) >= 2:
        E_star = rule[len(rule) // 2][3]

        def at(rows):
            Es = np.log([r[3] for r in rows])
            errs = np.log([max(r[2], 1e-300) for r in rows])
            order = np.argsort(Es)
            return float(np.exp(np.interp(math.log(E_star), Es[order], errs[order])))

        out.update({"E_bound": E_star, "rule_err_at_bound": at(rule), "learned_err_at_bound": at(learned),
                    "learned_brackets_bound": min(r[3] for r in learned) <= E_star <= max(r[3] for r in learned)})
    return out


def run(nx, ny, nz, U0, Re_f, mach, spinup, nsteps, stride, lambdas, precision, cfl, seed, flux="central",
        sep_steps=0, sens_lambdas=(), fd_eps=(0.05, 0.1, 0.2), judge=False, fd_steps=0,
        judge_rule=(0.2, 0.4, 0.8, 1.6, 2.4), judge_kappas=(0.2, 0.4, 0.8, 1.6, 3.2, 6.4, 12.8), judge_cap=False):
    gamma = 1.4
    dx = synth.box_shape(nx, ny, nz)
    Ly = ny * dx[1]
    mu = U0 * Ly / Re_f
    amp = synth.kolmogorov_amplitude(U0, mu, Ly)
    # start on the laminar profile the forcing sustains: its shear instability then grows
    # from the noise at inviscid rates instead of the profile building up on the viscous
    # time scale L_y^2 / nu
    w0 = synth.forced_start(nx, ny, nz, mach=mach, shear=U0, seed=seed, gamma=gamma)
    s_h = synth.kolmogorov_forcing(nx, ny, nz, amp)
    pt_in = (1.0 / gamma) * (1.0 + 0.5 * (gamma - 1.0) * mach ** 2) ** (gamma / (gamma - 1.0))
    S = api.Solver(nx, ny, nz, dx, gamma=gamma, mu=mu, Pr=0.72, dt=0.0, precision=precision,
                   plane_i=(3 * nx) // 4, pt_in=pt_in,
                   flux=api.NS_FLUX_ROE if flux == "roe" else api.NS_FLUX_CENTRAL)
    w = torch.from_numpy(w0).cuda()
    s = torch.from_numpy(s_h).cuda()
    # dt from the largest wave speed the developed flow is expected to reach (the stream
    # plus twice the laminar amplitude), at the given CFL number
    dt = cfl * min(dx) / (1.0 + mach + 2.0 * U0)
    S.set_dt(dt)
    t0 = time.perf_counter()
    a, b = w.clone(), torch.empty_like(w)
    history = []
    for n in range(spinup):
        S.primal_step(a, b, s)
        a, b = b, a
        if (n + 1) % max(1, spinup // 10) == 0:
            u = a[1:4] / a[0]
            # kinetic energy of the cross-stream velocity: zero on the laminar profile
            ke = float(0.5 * (a[0] * (u[1] ** 2 + u[2] ** 2)).mean())
            history.append({"step": n + 1, "cross_stream_kinetic_energy": ke})
    torch.cuda.synchronize()
    t_spin = time.perf_counter() - t0
    m = torch.empty(1, dtype=torch.float64, device="cuda")
    S.max_wave_speed(a, m)
    wspun = a.contiguous()
    out = {"box": [nx, ny, nz], "flux": flux, "mu": mu, "forcing_amplitude": amp, "U0": U0, "Re_f": Re_f, "mach": mach,
           "dt": dt, "cfl_at_spun_state": dt * m.item() / min(dx), "spinup_steps": spinup,
           "spinup_seconds": t_spin, "spinup_history": history, "finite": bool(torch.isfinite(wspun).all())}
    if not out["finite"]:
        return out
    if sep_steps:
        sep = separation(S, wspun, s, sep_steps)
        out["separation"] = sep
        # e-folds per step of the separation's growth over the second half of the record
        h = sep[len(sep) // 2:]
        if len(h) >= 2 and h[0][1] > 0 and h[-1][1] > 0:
            out["separation_efolds_per_step"] = math.log(h[-1][1] / h[0][1]) / (h[-1][0] - h[0][0])
    if sens_lambdas or judge:
        t0 = time.perf_counter()
        out["finite_differences"] = finite_differences(S, wspun, s, fd_steps or nsteps, fd_eps)
        out["finite_differences"]["seconds"] = time.perf_counter() - t0
    if sens_lambdas:
        out["sensitivity"] = sensitivity_scan(S, wspun, s, nsteps, stride, sens_lambdas, dx[0])
    if judge:
        S64 = api.Solver(nx, ny, nz, dx, gamma=gamma, mu=mu, Pr=0.72, dt=dt, precision=api.NS_FP64,
                         plane_i=(3 * nx) // 4, pt_in=pt_in,
                         flux=api.NS_FLUX_ROE if flux == "roe" else api.NS_FLUX_CENTRAL)
        out["closure_judge"] = closure_judge(S, S64, wspun, s, nsteps, stride, dx[0], judge_rule, judge_kappas,
                                             out["finite_differences"]["mean_dJ_dtheta"], cap=judge_cap)
        del S64
    # the plain adjoint from the developed state
    opts = S.run_opts(nsteps, api.NS_CKPT_STRIDE, stride, 0.0, 0.0, True, True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty_like(wspun)
    E = torch.zeros((nsteps + 1, 1), dtype=torch.float64, device="cuda")
    sig = torch.zeros((nsteps, 1, 2), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.adjoint_run(wspun, opts, arena, J, lam0, s=s, energy=E, sigma_stats=sig)
    torch.cuda.synchronize()
    Eh = E.cpu().numpy()[:, 0]
    sh = sig.cpu().numpy()[:, 0, :]
    norm = [float(Eh[nsteps - m] / (m + 1) ** 2) for m in (0, nsteps // 4, nsteps // 2, 3 * nsteps // 4, nsteps)]
    out.update({"nsteps": nsteps, "adjoint_seconds": time.perf_counter() - t0, "J_bar": float(J.item()),
                "E_normalised_at_m": dict(zip(["0", "N/4", "N/2", "3N/4", "N"], norm)),
                "efolds": api.energy_efolds(E.cpu().numpy(), nsteps, 1)[0],
                "sigma1_max_range": [float(sh[:, 0].min()), float(sh[:, 0].max())],
                "sigma1_mean_range": [float(sh[:, 1].min()), float(sh[:, 1].max())],
                "sticky_error": S.last_error()})
    if lambdas:
        lam_coefs = [t * dx[0] ** 2 for t in lambdas]
        opts = S.run_opts(nsteps, api.NS_CKPT_STRIDE, stride)
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
        work = torch.empty(S.estimate_work_bytes(opts), dtype=torch.uint8, device="cuda")
        t0 = time.perf_counter()
        chosen, ef, ch = S.estimate_lambda(wspun, opts, lam_coefs, arena, work, s=s)
        out.update({"lambda_tilde": list(lambdas), "lambda_efolds": ef, "lambda_change": ch,
                    "chosen_index": chosen, "chosen_lambda_tilde": lambdas[chosen] if chosen >= 0 else None,
                    "lambda_seconds": time.perf_counter() - t0, "sticky_error_lambda": S.last_error()})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--nx", type=int, default=128)
    ap.add_argument("--ny", type=int, default=64)
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--U0", type=float, default=0.3)
    ap.add_argument("--Re-f", type=float, default=2000.0)
    ap.add_argument("--mach", type=float, default=0.3)
    ap.add_argument("--spinup", type=int, default=6000)
    ap.add_argument("--nsteps", type=int, default=2000)
    ap.add_argument("--stride", type=int, default=50)
    ap.add_argument("--lambdas", default="")
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--cfl", type=float, default=0.5)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--flux", default="central", choices=["central", "roe"])
    ap.add_argument("--separation", type=int, default=0,
                    help="steps of the twin primal run that measures perturbation growth")
    ap.add_argument("--sens-lambdas", default="",
                    help="lambda-tilde values of the forcing-amplitude sensitivity scan against finite differences")
    ap.add_argument("--fd-eps", default="0.05,0.1,0.2")
    ap.add_argument("--fd-steps", type=int, default=0, help="horizon of the finite differences (default: nsteps)")
    ap.add_argument("--judge", action="store_true",
                    help="train the learned closure on this flow and judge it against the sigma_1 rule")
    ap.add_argument("--judge-rule", default="0.2,0.4,0.8,1.6,2.4", help="lambda-tilde values of the rule's sweep")
    ap.add_argument("--judge-kappas", default="0.2,0.4,0.8,1.6,3.2,6.4,12.8", help="kappa values of the learned sweep")
    ap.add_argument("--judge-cap", action="store_true",
                    help="hold both closures' coefficients at the explicit stability limit")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    lambdas = tuple(float(t) for t in a.lambdas.split(",")) if a.lambdas else ()
    res = run(a.nx, a.ny, a.nz, a.U0, a.Re_f, a.mach, a.spinup, a.nsteps, a.stride, lambdas,
              api.NS_FP64 if a.fp64 else api.NS_MIXED, a.cfl, a.seed, a.flux, a.separation,
              tuple(float(t) for t in a.sens_lambdas.split(",")) if a.sens_lambdas else (),
              tuple(float(t) for t in a.fd_eps.split(",")), a.judge, a.fd_steps,
              tuple(float(t) for t in a.judge_rule.split(",")), tuple(float(t) for t in a.judge_kappas.split(",")),
              a.judge_cap)
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()

"""Learned adjoint-viscosity closure: training data from this solver's own adjoints,
training with the library's BF16 kernels, and a judge against the plain sigma_1 rule.

The paper stabilises the unsteady adjoint by adding div(lambda sigma_1 grad w_hat) with
one hand-tuned lambda (section "Energy analysis", Table 2) and leaves the estimation of
lambda open.  The closure predicts a per-cell coefficient instead,
    nu(x) = kappa dx^2 sigma_1(x) softplus(MLP(f(x))),
trained on a label that balances, cell by cell, the growth and the dissipation terms of
the adjoint energy equation (Eq. e:energy_1) along short-horizon FP64 adjoints:
    t(x) = min(nu*(x) / (dx^2 sigma_1(x)), t_max),   nu* = max(0, v^T M v) / |grad v|^2.
Every numerical step runs in the CUDA library; this module only orchestrates calls and
holds memory.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import api

NIN, NH = 14, 64
PARAM_SHAPES = [("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)),
                ("b3", ())]


def pack(params: dict) -> np.ndarray:
    """Flat float32 parameter vector in the library's order."""
    return np.concatenate([np.asarray(params[k], dtype=np.float64).reshape(-1)
                           for k, _ in PARAM_SHAPES]).astype(np.float32)


def unpack(flat) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for k, shp in PARAM_SHAPES:
        n = int(np.prod(shp)) if shp else 1
        out[k] = flat[o:o + n].reshape(shp) if shp else flat[o]
        o += n
    return out


def init_params(seed: int = 0, out_bias: float = 0.0) -> dict:
    """He-style initialisation; out_bias sets softplus(b3) as the initial prediction."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return {
        "W1": rng.standard_normal((NIN, NH)) * math.sqrt(2.0 / NIN),
        "b1": np.zeros(NH),
        "W2": rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH),
        "b2": np.zeros(NH),
        "w3": rng.standard_normal(NH) * math.sqrt(0.1 / NH),
        "b3": out_bias,
    }


class Network:
    """A network blob on the device plus the calls that set, read and train it."""

    def __init__(self, solver: api.Solver, params: dict | None = None, seed: int = 0):
        self.S = solver
        self.blob = torch.zeros(api.mlp_net_bytes(), dtype=torch.uint8, device="cuda")
        self.step = 0
        self.set(params if params is not None else init_params(seed))

    def set(self, params: dict):
        flat = torch.from_numpy(pack(params)).cuda()
        self.S.mlp_set_params(self.blob, flat)
        self.step = 0

    def get(self) -> dict:
        out = torch.empty(api.NS_MLP_PARAMS, dtype=torch.float32, device="cuda")
        self.S.mlp_get_params(self.blob, out)
        return unpack(out.cpu().numpy())

    def train(self, feat: torch.Tensor, target: torch.Tensor, steps: int, batch: int = 4096,
              lr: float = 1e-3, seed: int = 0):
        """Adam steps on minibatches drawn with a seeded host generator (the draws are
        inputs of the kernels).  Returns the minibatch losses."""
        n = target.numel()
        rng = np.random.Generator(np.random.PCG64(seed))
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        losses = []
        for _ in range(steps):
            idx = torch.from_numpy(rng.integers(0, n, size=batch, dtype=np.int32)).cuda()
            self.step += 1
            self.S.mlp_train_step(self.blob, feat, target, idx, self.step, lr, loss)
            losses.append(loss)
            loss = torch.empty(1, dtype=torch.float32, device="cuda")
        return torch.cat(losses).cpu().numpy()


@dataclasses.dataclass
class Samples:
    feat: torch.Tensor      # [n, 16] float32
    target: torch.Tensor    # [n] float32


def trajectory(S: api.Solver, w0: torch.Tensor, nsteps: int, s: torch.Tensor | None = None):
    ws = [w0]
    for _ in range(nsteps):
        nxt = torch.empty_like(w0)
        S.primal_step(ws[-1], nxt, s)
        ws.append(nxt)
    return ws


def generate_samples(S: api.Solver, w0: torch.Tensor, nsteps: int, every: int = 4,
                     t_max: float = 10.0, s: torch.Tensor | None = None) -> Samples:
    """Run the unstabilised adjoint of the pressure loss over nsteps (all states kept,
    the primal driven by the source s if given) and, every `every` steps, pair the
    features of every cell of w^n with the label of (w^n, lam^n)."""
    ws = trajectory(S, w0, nsteps, s)
    cells = S.cells * S.batch
    lam = torch.zeros_like(w0)
    J = torch.zeros(S.batch, dtype=torch.float64, device=w0.device)
    S.objective(ws[nsteps], J, 1.0 / nsteps, lam)
    feats, targets = [], []
    sig = torch.empty(cells, dtype=torch.float32, device=w0.device)
    for n in range(nsteps - 1, -1, -1):
        nl = torch.empty_like(lam)
        S.adjoint_step(ws[n], lam, nl)
        lam = nl
        if n >= 1:
            S.objective(ws[n], J, 1.0 / nsteps, lam)
        if n % every == 0:
            acc = torch.zeros(cells, dtype=torch.float32, device=w0.device)
            S.adjoint_label(ws[n], lam, acc)
            S.growth_sigma1(ws[n], sig)
            feat = torch.empty((cells, 16), dtype=torch.float32, device=w0.device)
            S.mlp_features(ws[n], feat)
            t = torch.empty(cells, dtype=torch.float32, device=w0.device)
            S.label_target(acc, sig, t_max, t)
            feats.append(feat)
            targets.append(t)
    return Samples(torch.cat(feats).contiguous(), torch.cat(targets).contiguous())


# ----------------------------------------------------------------------------------
# the judge: sensitivity error against the exact short-horizon adjoint at matched
# adjoint energy, learned closure versus the sigma_1 rule
# ----------------------------------------------------------------------------------
def source_sensitivity(S: api.Solver, w0, phi, nsteps, lam_coef=0.0, mlp=None):
    """dJbar/dtheta for the source s = sum theta_m phi_m on x-momentum (theta = 0), and
    the adjoint energy E_vhat(w^0, lam^0), for one closure setting."""
    opts = S.run_opts(nsteps, api.NS_CKPT_ALL, 0, lam_coef, 0.0, True, False, mlp)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(S.batch, dtype=torch.float64, device="cuda")
    lam0 = torch.empty_like(w0)
    sbar = torch.empty_like(w0)
    E = torch.zeros((nsteps + 1, S.batch), dtype=torch.float64, device="cuda")
    S.adjoint_run(w0, opts, arena, J, lam0, sbar=sbar, energy=E)
    g = torch.empty(phi.shape[0], dtype=torch.float64, device="cuda")
    S.dot_boxes(sbar, 1, phi, g)
    return g.cpu().numpy(), float(E[0].sum().item()), float(E[:, 0].max().item())


def judge(S: api.Solver, w0, phi, nsteps, net: Network, rule_coefs, kappas):
    """Relative gradient error of each closure along its coefficient sweep and the error
    of each at the same adjoint-energy level (log-linear interpolation), with the energy
    of the rule's middle stable coefficient as the bound.  Settings that the library
    flags as beyond the explicit stability limit of the added viscosity are dropped."""
    g_exact, E_exact, _ = source_sensitivity(S, w0, phi, nsteps)
    if S.last_error() != 0:
        raise RuntimeError("the unstabilised reference adjoint raised a device error")
    nrm = np.linalg.norm(g_exact)

    def sweep(coefs, mlp):
        rows, dropped = [], []
        for c in coefs:
            g, E0, Emax = source_sensitivity(S, w0, phi, nsteps, c, mlp)
            if S.last_error() != 0 or not np.all(np.isfinite(g)):
                dropped.append(c)
                continue
            rows.append((c, float(np.linalg.norm(g - g_exact) / nrm), E0, Emax))
        return rows, dropped

    rule, rule_dropped = sweep(rule_coefs, None)
    learned, learned_dropped = sweep(kappas, net.blob)
    if len(rule) < 2 or len(learned) < 2:
        raise RuntimeError("too few stable settings in a sweep")
    E_star = rule[len(rule) // 2][2]

    def at(rows):
        Es = np.log([r[2] for r in rows])
        errs = np.log([max(r[1], 1e-300) for r in rows])
        order = np.argsort(Es)
        return float(np.exp(np.interp(math.log(E_star), Es[order], errs[order])))

    def brackets(rows):
        Es = [r[2] for r in rows]
        return min(Es) <= E_star <= max(Es)

    return {"E_exact": E_exact, "E_bound": E_star, "rule": rule, "learned": learned,
            "rule_dropped_unstable": rule_dropped, "learned_dropped_unstable": learned_dropped,
            "learned_brackets_bound": brackets(learned),
            "rule_err_at_bound": at(rule), "learned_err_at_bound": at(learned)}

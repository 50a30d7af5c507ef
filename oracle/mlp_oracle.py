"""Plain CPU oracle of the learned adjoint-viscosity closure.

TEST INFRASTRUCTURE ONLY (imported by tests/, never by the product path).  It shares no
code with the CUDA path.

The closure replaces the constant lambda of the stabilised adjoint equation (section
"Energy analysis": the added term div(lambda sigma_1 grad w_hat), with lambda tuned by
hand in the paper and its automatic estimation left as future work in the conclusion)
by a per-cell coefficient predicted from local flow features:

    nu(x) = dx^2 sigma_1(x) softplus(MLP(f(x)))

  * features f (14): the symmetrised variables v = S(q_bar)(q - q_bar) about the box-mean
    primitive state q_bar (section "Symmetrization", S of q_bar), divided by the mean
    sound speed c_bar, and the 9 entries of the velocity gradient (central differences)
    times L / c_bar with L = 1;
  * MLP: 14 -> 64 -> 64 -> 1, GELU hidden layers, softplus output; weights are BF16,
    accumulation FP32, hidden activations rounded to BF16 before the next layer (the
    tensor-core data path);
  * label (the paper has none): the local viscosity that balances the growth and the
    dissipation terms of Eq. (e:energy_1) for an added viscosity acting as an identity
    Laplacian on v_hat: nu* = max(0, v_hat^T M v_hat) / |grad v_hat|^2, time-averaged
    over an adjoint run and expressed as the coefficient t = nu* / (dx^2 sigma_1).

BF16 rounding is round-to-nearest-even of the float32 value to its top 16 bits.
"""
from __future__ import annotations

import math

import numpy as np

from . import ns_oracle as O

NIN, NH = 14, 64


# ----------------------------------------------------------------------------------
# BF16 rounding
# ----------------------------------------------------------------------------------
def bf16(x):
    """Round float values to bfloat16 (nearest, ties to even); returns float64 holding
    exactly representable bfloat16 values.  NaN/inf pass through."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) & 0xFFFF0000
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    special = ~np.isfinite(f)
    if np.any(special):
        out = np.where(special, f.astype(np.float64), out)
    return out


# ----------------------------------------------------------------------------------
# activations
# ----------------------------------------------------------------------------------
_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def softplus(y):
    return np.maximum(y, 0.0) + np.log1p(np.exp(-np.abs(y)))


def softplus_grad(y):
    return 1.0 / (1.0 + np.exp(-y))


# ----------------------------------------------------------------------------------
# parameters
# ----------------------------------------------------------------------------------
def init_params(seed=0):
    """W1[14,64], b1[64], W2[64,64], b2[64], w3[64], b3 (float64, He-like scaling)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((NIN, NH)) * math.sqrt(2.0 / NIN),
        "b1": np.zeros(NH),
        "W2": rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH),
        "b2": np.zeros(NH),
        "w3": rng.standard_normal(NH) * math.sqrt(1.0 / NH),
        "b3": np.array(0.0),
    }


def forward(p, X, quantize=True):
    """Forward pass on X[n,14].  quantize=True applies the BF16 data path (weights and
    inputs of each matrix product rounded to BF16, products summed exactly / in FP64
    here); quantize=False is the plain FP64 network.  Returns output y (pre-softplus),
    prediction softplus(y) and the cache for backward."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    X0 = q(X)
    Z1 = X0 @ q(p["W1"]) + p["b1"]
    H1 = gelu(Z1)
    H1q = q(H1)
    Z2 = H1q @ q(p["W2"]) + p["b2"]
    H2 = gelu(Z2)
    y = H2 @ q(p["w3"]) + p["b3"]
    cache = dict(X0=X0, Z1=Z1, H1q=H1q, Z2=Z2, H2=H2, y=y)
    return y, softplus(y), cache


def loss_and_grads(p, X, t, quantize=True, bf16_backward=False):
    """Mean squared error of softplus(MLP(X)) against targets t and its gradient with
    respect to every parameter (hand-derived backward; the BF16 rounding points are
    treated as identity in the backward pass, the usual straight-through rule).
    bf16_backward=True also rounds the pre-activation gradients dZ2 and dZ1 to BF16
    where they enter matrix products (the weight gradients and dH1), the data path of
    a BF16 tensor-core backward pass; the bias gradients sum the unrounded ones."""
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    n = X.shape[0]
    y, pred, c = forward(p, X, quantize)
    r = pred - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / n * softplus_grad(y)
    g = {}
    g["w3"] = c["H2"].T @ dy
    g["b3"] = np.array(np.sum(dy))
    dH2 = np.outer(dy, q(p["w3"]))
    dZ2 = dH2 * gelu_grad(c["Z2"])
    dZ2m = bf16(dZ2) if bf16_backward else dZ2      # operand of the products below
    g["W2"] = c["H1q"].T @ dZ2m
    g["b2"] = np.sum(dZ2, axis=0)
    dH1 = dZ2m @ q(p["W2"]).T
    dZ1 = dH1 * gelu_grad(c["Z1"])
    dZ1m = bf16(dZ1) if bf16_backward else dZ1
    g["W1"] = c["X0"].T @ dZ1m
    g["b1"] = np.sum(dZ1, axis=0)
    return L, g


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, bias-corrected) of the FP64 master parameters."""
    out_p, out_m, out_v = {}, {}, {}
    for k in p:
        out_m[k] = b1 * m[k] + (1 - b1) * g[k]
        out_v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = out_m[k] / (1 - b1 ** step)
        vh = out_v[k] / (1 - b2 ** step)
        out_p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return out_p, out_m, out_v


# ----------------------------------------------------------------------------------
# features and label
# ----------------------------------------------------------------------------------
def features(w, P: O.Params):
    """f[cells, 14] of one box (see module docstring)."""
    g = P.gamma
    rho, u, e, p = O.primitives(w, P)
    rb, ub, pb = rho.mean(), u.mean(axis=(1, 2, 3)), p.mean()
    cb = math.sqrt(g * pb / rb)
    v = np.empty((5,) + rho.shape)
    v[0] = cb / (math.sqrt(g) * rb) * (rho - rb)
    for k in range(3):
        v[1 + k] = u[k] - ub[k]
    v[4] = (-cb / (rb * math.sqrt(g * (g - 1))) * (rho - rb)
            + math.sqrt(g / (g - 1)) / (rb * cb) * (p - pb))
    f = [v[i] / cb for i in range(5)]
    for k in range(3):
        for j in range(3):
            f.append(O._central(u[k], j, P) / cb)
    return np.stack([a.ravel() for a in f], axis=1)


def label_rate(w, lam, P: O.Params, eps=1e-30):
    """Per-cell growth / dissipation balance of one adjoint state: with v_hat = T^-T lam,
    nu* = max(0, v_hat^T M v_hat) / |grad v_hat|^2 (central differences of every
    component).  For a 2D box the (rho, u1, u2, p) block of M and v_hat is used, as for
    sigma_1."""
    vh = O.symmetric_adjoint(w, lam, P)
    M = O.growth_matrix_field(w, P)
    if w.shape[1] == 1:
        idx = [0, 1, 2, 4]
        M = M[..., idx, :][..., :, idx]
        vh = vh[idx]
    vc = np.moveaxis(vh, 0, -1)
    growth = np.einsum("...i,...ij,...j->...", vc, M, vc)
    grad2 = np.zeros(w.shape[1:])
    for d in range(3):
        gd = (np.roll(vh, -1, axis=3 - d) - np.roll(vh, 1, axis=3 - d)) / (2.0 * P.dx[d])
        grad2 += np.sum(gd * gd, axis=0)
    return np.maximum(growth, 0.0) / (grad2 + eps)


def label_coefficient(nu_star_mean, sigma1, dx, eps=1e-30):
    """Training target t = nu* / (dx^2 sigma_1) from a time-averaged nu*."""
    return nu_star_mean / (dx * dx * sigma1 + eps)

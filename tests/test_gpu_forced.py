"""The forced-box study and the adjoint-energy series of a sweep (section "Energy
analysis": E_vhat of the stabilised adjoint; section "Results": the adjoint of a
turbulent flow and its growth)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1511_06959_gb300 import forced_study, synth
from tests.test_gpu_parity import _api, dev, host, make_solver
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
def test_sweep_energy_matches_the_standalone_energy(prec):
    """E[0] of a sweep (after the last reversed step) equals ns_adjoint_energy(w^0,
    lam^0): the same per-cell arithmetic on the same values (FP64, or the float
    roundings of w^0 and lam^0 that the sweep keeps as mirrors)."""
    api = _api()
    w0 = synth.isentropic_vortex(40, 24, 3, noise=1e-3, seed=8)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    S = make_solver(api, w0, P, prec)
    N = 7
    opts = S.run_opts(N, api.NS_CKPT_STRIDE, 3, 0.3 * P.dx[0] ** 2, 0.0, True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    E = torch.zeros((N + 1, 1), dtype=torch.float64, device="cuda")
    S.adjoint_run(dev(w0), opts, arena, J, lam0, energy=E)
    E0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.adjoint_energy(dev(w0), lam0, E0)
    assert S.last_error() == 0
    assert np.all(host(E) > 0.0)
    np.testing.assert_allclose(host(E)[0, 0], host(E0)[0], rtol=1e-12)


def test_forced_study_runs_on_a_small_box():
    """Spin-up, twin-run separation, the plain adjoint's growth, the lambda scan and the
    sensitivity scan against finite differences on a 32 x 16 x 8 forced box: every
    figure finite, and on this short horizon the adjoint's forcing sensitivity agrees
    with the finite difference."""
    res = forced_study.run(32, 16, 8, U0=0.3, Re_f=500.0, mach=0.3, spinup=30, nsteps=24, stride=6,
                           lambdas=(0.0, 0.4), precision=1, cfl=0.5, seed=5, sep_steps=20,
                           sens_lambdas=(0.0, 0.4), fd_eps=(0.1,))
    assert res["finite"] and res["sticky_error"] == 0
    assert all(math.isfinite(v) for _, v in res["separation"])
    assert math.isfinite(res["efolds"]) and len(res["lambda_efolds"]) == 2
    sens = res["sensitivity"]
    assert all(math.isfinite(r["dJ_dtheta"]) and r["sticky_error"] == 0 for r in sens["adjoint"])
    assert math.isfinite(res["finite_differences"]["mean_dJ_dtheta"])
    # the sweeps' J-bar does not depend on lambda
    assert abs(sens["J_bar"] - res["J_bar"]) <= 1e-12 * abs(res["J_bar"])
    # a short horizon is not chaotic: the unstabilised adjoint's dJ/dtheta = <s-bar, s>
    # is the derivative the central difference approximates (to O(eps^2))
    g_adj = sens["adjoint"][0]["dJ_dtheta"]
    g_fd = res["finite_differences"]["rows"][0]["dJ_dtheta"]
    assert abs(g_adj - g_fd) <= 0.05 * abs(g_fd)

"""The bounds-checking build (NS_DEBUG_BOUNDS): every field access of the stencil kernels
is checked against its field's extent and a wrong index is reported as NS_ERR_BOUNDS
instead of reaching memory.  On valid inputs it must change nothing: a subprocess that
loads the debug library (NS_ADJOINT_LIB) runs residuals, adjoint steps, a checkpointed
stabilised sweep, a bounded box and two slabs, and its results equal the release
library's bit for bit with a clear error word.  No out-of-range input is run here."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_1511_06959_gb300 import api, synth
from paper_1511_06959_gb300 import slabs as SL
from tests.test_oracle_primal import params_for

out = {}
def put(k, t):
    out[k] = t.detach().cpu().numpy().ravel().tolist()
for prec in (0, 1):
    w = synth.isentropic_vortex(37, 9, 5, noise=1e-3, seed=61)
    P = params_for(w, mu=1e-3, dt=3e-3)
    S = api.Solver(37, 9, 5, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt, precision=prec,
                   plane_i=P.plane_i, pt_in=P.pt_in)
    wd = torch.from_numpy(w).cuda()
    R = torch.empty_like(wd)
    S.rhs(wd, R)
    put(f"rhs{prec}", R)
    lam = torch.from_numpy(synth.random_field(w.shape, 62)).cuda()
    nu = torch.full(w.shape[1:], 1e-5, dtype=torch.float32, device="cuda")
    lo = torch.empty_like(wd)
    S.adjoint_step(wd, lam, lo, nu=nu)
    put(f"adj{prec}", lo)
    opts = S.run_opts(9, api.NS_CKPT_STRIDE, 3, 0.5 * P.dx[0] ** 2, 0.0, True, True, verify=True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty_like(wd)
    E = torch.empty((10, 1), dtype=torch.float64, device="cuda")
    S.adjoint_run(wd, opts, arena, J, lam0, energy=E)
    put(f"sweep{prec}", lam0)
    put(f"E{prec}", E)
    out[f"err{prec}"] = S.last_error()
    B = api.Solver(37, 9, 5, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt, precision=prec,
                   plane_i=P.plane_i, pt_in=P.pt_in)
    B.set_boundaries(api.NS_BC_INOUT_WALLS, far=(1.0, 0.5, 0.0, 0.0, 1.0 / 1.4), wall_e=(1.7, 1.9))
    lb = torch.empty_like(wd)
    B.adjoint_step(wd, lam, lb, nu=nu)
    put(f"bounded{prec}", lb)
    out[f"errb{prec}"] = B.last_error()
    cuts = [(0, 15), (15, 37)]
    Ss = [api.Solver(b - a + 2, 9, 5, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt, precision=prec)
          for a, b in cuts]
    G = api.SlabGroup(Ss)
    wk = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in SL.split(w, cuts)]
    ok = [torch.empty_like(t) for t in wk]
    G.primal_step(wk, ok)
    put(f"slab{prec}", SL.join(ok))
torch.cuda.synchronize()
print(json.dumps(out))
""".replace("ROOT", repr(ROOT))


def _run(lib):
    env = dict(os.environ)
    if lib:
        env["NS_ADJOINT_LIB"] = lib
    else:
        env.pop("NS_ADJOINT_LIB", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checking_build_changes_nothing_on_valid_inputs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_06959_gb300 import build
    if not os.path.exists(build.OUT):
        build.build()
    if not os.path.exists(build.OUT_DEBUG):
        build.build(debug=True)
    rel = _run(None)
    dbg = _run(build.OUT_DEBUG)
    for k, v in rel.items():
        if k.startswith("err"):
            assert v == 0 and dbg[k] == 0, (k, v, dbg[k])
        else:
            assert np.array_equal(np.array(v), np.array(dbg[k])), k

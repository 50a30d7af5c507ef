"""A sweep captured as one CUDA graph (ns_adjoint_run_capture / ns_graph_launch): every
replay does the whole sweep again and gives the bits of ns_adjoint_run on the inputs as
they are at replay time; the host and disk tiers are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, make_solver
from tests.test_gpu_sweep import _run
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu


def _outputs(S, w0, N):
    J = torch.full((S.batch,), float("nan"), dtype=torch.float64, device="cuda")
    lam0 = torch.full(w0.shape, float("nan"), dtype=torch.float64, device="cuda")
    sbar = torch.full_like(lam0, float("nan"))
    E = torch.full((N + 1, S.batch), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((N, S.batch, 2), float("nan"), dtype=torch.float64, device="cuda")
    return J, lam0, sbar, E, st


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("schedule,param", [(1, 4), (2, 3)])
def test_captured_sweep_replays_the_bits_of_the_direct_sweep(prec, schedule, param):
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N = 14
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, w0, P, prec)
    ref = _run(api, S, w0, N, schedule, param, s, lam_coef=lam_coef, energy=True, sigma=True)
    opts = S.run_opts(N, schedule, param, lam_coef, 0.0, True, True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    W0, SRC = dev(w0), dev(s)
    J, lam0, sbar, E, st = out = _outputs(S, w0, N)
    launches = api.launch_count()
    G = S.adjoint_run_capture(W0, opts, arena, J, lam0, s=SRC, sbar=sbar, energy=E, sigma_stats=st)
    torch.cuda.synchronize()
    # capture records the launches without running them
    assert torch.isnan(lam0).all() and torch.isnan(J).all()
    assert G.kernels == api.launch_count() - launches > 0
    for _ in range(2):
        for t in out:
            t.fill_(float("nan"))
        G.launch()
        torch.cuda.synchronize()
        assert S.last_error() == 0
        for got, want in zip(out, ref):
            assert torch.equal(got, want)
    G.close()


def test_replay_reads_the_inputs_at_replay_time():
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    w1 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=6)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    N = 9
    S = make_solver(api, w0, P, 1)
    opts = S.run_opts(N, 1, 4, 0.0, 0.0, True, True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    W0 = dev(w0)
    J, lam0, sbar, E, st = out = _outputs(S, w0, N)
    G = S.adjoint_run_capture(W0, opts, arena, J, lam0, sbar=sbar, energy=E, sigma_stats=st)
    W0.copy_(dev(w1))
    G.launch()
    torch.cuda.synchronize()
    ref = _run(api, S, w1, N, 1, 4, energy=True, sigma=True)
    assert torch.equal(J, ref[0]) and torch.equal(lam0, ref[1])
    assert torch.equal(E, ref[3]) and torch.equal(st, ref[4])
    # the solver's close releases its graphs first
    S.close()
    assert not G._g


def test_capture_refuses_the_host_and_disk_tiers(tmp_path):
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    S = make_solver(api, w0, P, 0)
    N = 9
    for sched, kw in [(api.NS_CKPT_STRIDE_HOST, {}), (api.NS_CKPT_STRIDE_DISK, {"disk_path": str(tmp_path / "s.bin")}),
                      (api.NS_CKPT_REVOLVE_HOST, {}), (api.NS_CKPT_REVOLVE_DISK, {"disk_path": str(tmp_path / "r.bin")})]:
        host = torch.zeros(max(S.host_bytes(S.run_opts(N, sched, 3)), 256), dtype=torch.uint8, pin_memory=True)
        if sched in (api.NS_CKPT_STRIDE_HOST, api.NS_CKPT_REVOLVE_HOST):
            kw = {"host_arena": host}
        opts = S.run_opts(N, sched, 3, **kw)
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
        J, lam0, _, _, _ = _outputs(S, w0, N)
        with pytest.raises(api.NsError) as e:
            S.adjoint_run_capture(dev(w0), opts, arena, J, lam0)
        assert e.value.code == api.NS_ERR_ARG
    # the context still runs a direct sweep afterwards
    ref = _run(api, S, w0, N, 1, 3)
    assert torch.isfinite(ref[1]).all()

"""x-slab decomposition on one GPU: slab contexts over padded slabs, stepped together by
ns_slab_* with their ghost columns exchanged after every stage, give the unsplit box's
states, objective and adjoint bit for bit in their interior columns, over a short
sweep (primal steps, the time-averaged objective, the adjoint steps with the objective
source and, optionally, the added viscosity)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1511_06959_gb300 import slabs as SL
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, make_solver
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu

NX, NY, NZ, N = 32, 10, 4, 5


def _slab_solvers(api, P, cuts, prec, plane, streams=None):
    out = []
    for k, (a, b) in enumerate(cuts):
        # the objective plane's two columns must be interior to the slab that evaluates it
        pi = plane - a + 1 if a < plane <= b - 1 else 1
        out.append(api.Solver(b - a + 2, NY, NZ, P.dx, gamma=P.gamma, mu=P.mu, Pr=P.Pr, dt=P.dt, precision=prec,
                              plane_i=pi, pt_in=P.pt_in, stream=None if streams is None else streams[k]))
    return out


def _owner(cuts, plane):
    return [k for k, (a, b) in enumerate(cuts) if a < plane <= b - 1][0]


def _sweep_full(api, S, w0, lam_coef):
    """N steps, Jbar and dJbar/dw0 of the unsplit box (the right-endpoint mean)."""
    ws = [dev(w0)]
    for n in range(N):
        w1 = torch.empty_like(ws[0])
        S.primal_step(ws[-1], w1)
        ws.append(w1)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(1, N + 1):
        S.objective(ws[n], J, 1.0 / N)
    lam = torch.zeros_like(ws[0])
    S.objective(ws[N], torch.zeros_like(J), 1.0 / N, lam)
    for n in range(N - 1, -1, -1):
        nu = None
        if lam_coef > 0:
            sig = torch.empty(ws[0].shape[-3:], dtype=torch.float32, device="cuda")
            S.growth_sigma1(ws[n], sig)
            nu = torch.empty_like(sig)
            S.add_adjoint_viscosity(sig, lam_coef, nu)
        lo = torch.empty_like(lam)
        S.adjoint_step(ws[n], lam, lo, nu=nu)
        lam = lo
        if n >= 1:
            S.objective(ws[n], torch.zeros_like(J), 1.0 / N, lam)
    torch.cuda.synchronize()
    return ws, J, lam


def _sweep_slabs(api, G, Ss, wk0, own, lam_coef):
    K = len(Ss)
    ws = [[dev(w) for w in wk0]]
    for n in range(N):
        out = [torch.empty_like(t) for t in ws[-1]]
        G.primal_step(ws[-1], out)
        ws.append(out)
    torch.cuda.synchronize()
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in range(1, N + 1):
        Ss[own].objective(ws[n][own], J, 1.0 / N)
    lam = [torch.zeros_like(t) for t in ws[0]]
    Ss[own].objective(ws[N][own], torch.zeros_like(J), 1.0 / N, lam[own])
    G.exchange(lam, 5)
    for n in range(N - 1, -1, -1):
        nu = None
        if lam_coef > 0:
            nu = []
            for k in range(K):
                sig = torch.empty(ws[0][k].shape[-3:], dtype=torch.float32, device="cuda")
                Ss[k].growth_sigma1(ws[n][k], sig)
                v = torch.empty_like(sig)
                Ss[k].add_adjoint_viscosity(sig, lam_coef, v)
                nu.append(v)
            G.exchange(nu, 1)
        lo = [torch.empty_like(t) for t in lam]
        G.adjoint_step(ws[n], lam, lo, nu=nu)
        lam = lo
        if n >= 1:
            Ss[own].objective(ws[n][own], torch.zeros_like(J), 1.0 / N, lam[own])
            G.exchange(lam, 5)
    torch.cuda.synchronize()
    return ws, J, lam


@pytest.mark.parametrize("prec,lam_tilde,cuts", [
    (0, 0.0, [(0, 13), (13, 32)]),
    (1, 0.0, [(0, 13), (13, 32)]),
    (0, 0.5, [(0, 11), (11, 20), (20, 32)]),
    (1, 0.5, [(0, 11), (11, 20), (20, 32)]),
])
def test_slabs_equal_the_unsplit_box_bitwise(prec, lam_tilde, cuts):
    api = _api()
    w0 = synth.isentropic_vortex(NX, NY, NZ, noise=1e-3, seed=9)
    P = params_for(w0, mu=1e-3, dt=3e-3)
    lam_coef = lam_tilde * P.dx[0] ** 2
    S = make_solver(api, w0, P, prec)
    ws, J, lam0 = _sweep_full(api, S, w0, lam_coef)
    Ss = _slab_solvers(api, P, cuts, prec, P.plane_i)
    G = api.SlabGroup(Ss)
    wk, Jk, lamk = _sweep_slabs(api, G, Ss, SL.split(w0, cuts), _owner(cuts, P.plane_i), lam_coef)
    for n in range(N + 1):
        assert torch.equal(SL.join(wk[n]), ws[n]), n
    assert torch.equal(Jk, J)
    assert torch.equal(SL.join(lamk), lam0)
    # the ghost columns hold the neighbours' boundary columns after every call
    for k, (a, b) in enumerate(cuts):
        cols = SL.padded_columns(NX, a, b)
        assert torch.equal(lamk[k], lam0[..., cols])
    for s in Ss:
        assert s.last_error() == 0


def test_slabs_on_separate_streams():
    """Each slab context on its own stream: the exchanges order the streams with events."""
    api = _api()
    w0 = synth.isentropic_vortex(NX, NY, NZ, noise=1e-3, seed=10)
    P = params_for(w0, mu=1e-3, dt=3e-3)
    cuts = SL.cuts_even(NX, 3)
    S = make_solver(api, w0, P, 1)
    ws, J, lam0 = _sweep_full(api, S, w0, 0.0)
    streams = [torch.cuda.Stream() for _ in cuts]
    Ss = _slab_solvers(api, P, cuts, 1, P.plane_i, streams)
    G = api.SlabGroup(Ss)
    wk = [dev(w) for w in SL.split(w0, cuts)]
    torch.cuda.synchronize()
    for n in range(N):
        out = [torch.empty_like(t) for t in wk]
        torch.cuda.synchronize()
        G.primal_step(wk, out)
        torch.cuda.synchronize()
        wk = out
    assert torch.equal(SL.join(wk), ws[N])


def test_one_slab_with_a_host_exchange_hook():
    """A one-slab group whose ghosts a host function fills (the path of one slab per
    process, here with the slab its own periodic neighbour) gives the unsplit box."""
    api = _api()
    w0 = synth.isentropic_vortex(NX, NY, NZ, noise=1e-3, seed=11)
    P = params_for(w0, mu=1e-3, dt=3e-3)
    S = make_solver(api, w0, P, 0)
    ws, J, lam0 = _sweep_full(api, S, w0, 0.0)
    (S1,) = _slab_solvers(api, P, [(0, NX)], 0, P.plane_i)
    calls = []

    hook = SL.halo_exchange_fn(S1, rank=0, world=1)

    def counted(ptr, eb, nc):
        calls.append((eb, nc))
        return hook(ptr, eb, nc)

    G = api.SlabGroup([S1], exchange=counted)
    wk, Jk, lamk = _sweep_slabs(api, G, [S1], SL.split(w0, [(0, NX)]), 0, 0.0)
    assert torch.equal(SL.join(wk[N]), ws[N])
    assert torch.equal(Jk, J)
    assert torch.equal(SL.join(lamk), lam0)
    # four stage outputs per primal step; three recomputed stages and four seeds per
    # adjoint step; the objective's scatter N times
    assert len(calls) == 4 * N + 7 * N + N


@pytest.mark.parametrize("prec,lam_tilde", [(0, 0.0), (1, 0.5)])
@pytest.mark.parametrize("sched", [(0, 0), (1, 2), (2, 2)])
def test_slab_checkpointed_sweep(prec, lam_tilde, sched):
    """ns_slab_adjoint_run (store-all, stride and revolve plans executed on every slab,
    states kept per slab) gives the bits of the same slab calls made step by step, and so
    the unsplit box's J-bar and dJ-bar/dw0 in every interior column."""
    api = _api()
    w0 = synth.isentropic_vortex(NX, NY, NZ, noise=1e-3, seed=10)
    P = params_for(w0, mu=1e-3, dt=3e-3)
    cuts = [(0, 13), (13, 32)]
    lam_coef = lam_tilde * P.dx[0] ** 2
    Ss = _slab_solvers(api, P, cuts, prec, P.plane_i)
    G = api.SlabGroup(Ss)
    own = _owner(cuts, P.plane_i)
    wk0 = [dev(w) for w in SL.split(w0, cuts)]
    _, Jref, lamref = _sweep_slabs(api, G, Ss, SL.split(w0, cuts), own, lam_coef)
    schedule, param = sched
    opts = Ss[0].run_opts(N, schedule, param, lam_coef)
    work = [torch.empty(b, dtype=torch.uint8, device="cuda") for b in G.run_bytes(opts)]
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = [torch.empty_like(w) for w in wk0]
    G.adjoint_run(own, wk0, opts, work, J, lam0)
    torch.cuda.synchronize()
    assert all(S.last_error() == 0 for S in Ss)
    assert torch.equal(J, Jref)
    for a, b in zip(lam0, lamref):
        assert torch.equal(a, b)
    # the unsplit box
    S = make_solver(api, w0, P, prec)
    _, Jf, lamf = _sweep_full(api, S, w0, lam_coef)
    assert torch.equal(J, Jf)
    assert torch.equal(SL.join(lam0), lamf)
    # the host tier and a short workspace are refused
    with pytest.raises(api.NsError):
        G.adjoint_run(own, wk0, Ss[0].run_opts(N, api.NS_CKPT_STRIDE_HOST, 2), work, J, lam0)
    short = [w[: w.numel() - 256] for w in work]
    with pytest.raises(api.NsError) as e:
        G.adjoint_run(own, wk0, opts, short, J, lam0)
    assert e.value.code == api.NS_ERR_BUDGET


def test_slab_group_arguments():
    api = _api()
    w0 = synth.isentropic_vortex(NX, NY, NZ, noise=0.0)
    P = params_for(w0, mu=1e-3, dt=3e-3)
    a = api.Solver(10, NY, NZ, P.dx, dt=P.dt)
    b = api.Solver(10, NY + 1, NZ, P.dx, dt=P.dt)
    with pytest.raises(api.NsError):
        api.SlabGroup([a, b])
    c = api.Solver(2, NY, NZ, P.dx, dt=P.dt)
    with pytest.raises(api.NsError):
        api.SlabGroup([a, c])
    with pytest.raises(api.NsError):
        api.SlabGroup([a, a], exchange=lambda p, e, n: 0)

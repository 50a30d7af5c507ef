"""GPU checkpointed sweep (ns_adjoint_run) against the oracle's store-all adjoint and
across schedules: replay is bitwise deterministic, so every schedule gives the same
bits; the added viscosity, sigma_1 statistics and the adjoint-energy series follow the
oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, host, make_solver, rel_l2
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu


def _run(api, S, w0, N, schedule, param, s=None, lam_coef=0.0, tau=0.0, energy=False, sigma=False):
    opts = S.run_opts(N, schedule, param, lam_coef, tau, energy, sigma)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(S.batch, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    sbar = torch.empty_like(lam0)
    E = torch.zeros((N + 1, S.batch), dtype=torch.float64, device="cuda") if energy else None
    st = torch.zeros((N, S.batch, 2), dtype=torch.float64, device="cuda") if sigma else None
    S.adjoint_run(dev(w0), opts, arena, J, lam0, s=None if s is None else dev(s), sbar=sbar,
                  energy=E, sigma_stats=st)
    torch.cuda.synchronize()
    return J, lam0, sbar, E, st


@pytest.mark.parametrize("prec", [0, 1])
def test_schedules_agree_bitwise_and_match_oracle(prec):
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N = 13
    S = make_solver(api, w0, P, prec)
    # stride 4, 5 and 20: a last segment of 1, 3 and all 13 steps, reversed from the
    # states and stage states the forward pass keeps
    res = [_run(api, S, w0, N, sch, prm, s) for sch, prm in [(0, 0), (1, 4), (1, 5), (1, 20), (2, 3), (2, 1)]]
    for J, lam, sb, _, _ in res[1:]:
        assert torch.equal(J, res[0][0])
        assert torch.equal(lam, res[0][1])
        assert torch.equal(sb, res[0][2])
    ws, Jref = O.primal_run(w0, P, N, s)
    lam_ref, sbar_ref = O.adjoint_run(ws, P, s)
    tol = 1e-10 if prec == 0 else 1e-4
    J, lam, sb, _, _ = res[0]
    assert abs(J.item() - Jref) <= tol * abs(Jref)
    assert rel_l2(host(lam), lam_ref) < tol
    assert rel_l2(host(sb), sbar_ref) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_pipelined_stride_sweep_gives_the_sequential_bits(prec):
    """A stride sweep of several segments replays the next segment on a second stream while
    it reverses the current one; with ns_set_pipeline off it runs them in sequence.  Both
    give the same bits (stabilised, with a source, energy and sigma_1 series), and the
    pipelined arena holds the second set of segment states and kept stages."""
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N, k = 23, 4
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, w0, P, prec)
    opts = S.run_opts(N, 1, k, lam_coef, 0.0, True, True)
    big = S.arena_bytes(opts)
    pipe = _run(api, S, w0, N, 1, k, s, lam_coef=lam_coef, energy=True, sigma=True)
    S.set_pipeline(False)
    assert S.arena_bytes(opts) < big
    seq = _run(api, S, w0, N, 1, k, s, lam_coef=lam_coef, energy=True, sigma=True)
    S.set_pipeline(True)
    again = _run(api, S, w0, N, 1, k, s, lam_coef=lam_coef, energy=True, sigma=True)
    assert S.last_error() == 0
    for a, b, c in zip(pipe, seq, again):
        assert torch.equal(a, b) and torch.equal(a, c)


def test_stabilised_sweep_energy_and_sigma_series():
    api = _api()
    w0 = synth.isentropic_vortex(40, 12, 1, noise=1e-3, seed=6)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    N = 9
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, w0, P)
    J, lam, sb, E, st = _run(api, S, w0, N, 2, 2, lam_coef=lam_coef, energy=True, sigma=True)
    assert S.last_error() == 0
    ws, Jref = O.primal_run(w0, P, N)
    nu_of = lambda w: lam_coef * O.sigma1_field(w, P)
    lam_ref, _ = O.adjoint_run(ws, P, None, nu_of)
    # FP64 context: sigma_1 and nu are carried in FP64 through the sweep
    assert rel_l2(host(lam), lam_ref) < 1e-10
    # energy series E(w^n, lam^n): recompute lam^n with the oracle sweep
    lam_n = np.zeros_like(w0)
    Eref = np.zeros(N + 1)
    lam_n = O.objective_grad(ws[N], P) / N
    Eref[N] = O.adjoint_energy(ws[N], lam_n, P)
    for n in range(N, 0, -1):
        lam_n, _ = O.rk4_adjoint_step(ws[n - 1], lam_n, P, None, nu_of(ws[n - 1]))
        if n - 1 >= 1:
            lam_n = lam_n + O.objective_grad(ws[n - 1], P) / N
        Eref[n - 1] = O.adjoint_energy(ws[n - 1], lam_n, P)
    np.testing.assert_allclose(host(E)[:, 0], Eref, rtol=1e-10)
    sig_ref = np.array([[O.sigma1_field(ws[n], P).max(), O.sigma1_field(ws[n], P).mean()]
                        for n in range(N)])
    np.testing.assert_allclose(host(st)[:, 0, :], sig_ref, rtol=1e-10)


def test_budget_too_small_is_reported():
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 1, noise=0.0)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    S = make_solver(api, w0, P)
    opts = S.run_opts(10, 0, 0)
    need = S.arena_bytes(opts)
    arena = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(api.NsError) as e:
        S.adjoint_run(dev(w0), opts, arena, J, lam0)
    assert e.value.code == api.NS_ERR_BUDGET


def test_batched_sweep_matches_single_boxes():
    api = _api()
    shape = (33, 8, 4)
    ws0 = np.stack([synth.isentropic_vortex(*shape, noise=1e-3, seed=20 + i) for i in range(3)])
    P = params_for(ws0[0], mu=1e-3, dt=4e-3)
    N = 6
    S = make_solver(api, ws0[0], P, batch=3)
    J, lam, _, _, _ = _run(api, S, ws0, N, 1, 2)
    S1 = make_solver(api, ws0[0], P)
    for i in range(3):
        Ji, li, _, _, _ = _run(api, S1, ws0[i], N, 1, 2)
        assert J[i].item() == Ji.item()
        assert torch.equal(lam[i], li[0] if li.dim() == 5 else li)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_sigma_and_energy_series_match_single_boxes(prec):
    """A batch of three boxes: each box's sigma_1 statistics (per-box partials of every
    CTA, reduced by the last one) and energy series equal the single box's, the maxima
    exactly and the sums to their summation order."""
    api = _api()
    shape = (33, 8, 4)
    ws0 = np.stack([synth.isentropic_vortex(*shape, noise=1e-3, seed=30 + i) for i in range(3)])
    P = params_for(ws0[0], mu=1e-3, dt=4e-3)
    N = 5
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, ws0[0], P, prec, batch=3)
    _, _, _, E, st = _run(api, S, ws0, N, 1, 2, lam_coef=lam_coef, energy=True, sigma=True)
    assert S.last_error() == 0
    S1 = make_solver(api, ws0[0], P, prec)
    for i in range(3):
        _, _, _, Ei, sti = _run(api, S1, ws0[i], N, 1, 2, lam_coef=lam_coef, energy=True, sigma=True)
        assert torch.equal(st[:, i, 0], sti[:, 0, 0])
        np.testing.assert_allclose(host(st[:, i, 1]), host(sti[:, 0, 1]), rtol=1e-12)
        np.testing.assert_allclose(host(E[:, i]), host(Ei[:, 0]), rtol=1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_host_snapshots_give_the_stride_bits(prec):
    """NS_CKPT_STRIDE_HOST keeps the every-k-th snapshots in host memory and copies them
    on the context's stream: the sweep (stabilised, with a source, energy and sigma_1
    series) gives the stride schedule's bits, from page-locked and from pageable host
    memory, in less device memory; a short host arena is a budget error."""
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N, k = 14, 4
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, w0, P, prec)
    ref = _run(api, S, w0, N, 1, k, s, lam_coef=lam_coef, energy=True, sigma=True)
    probe = S.run_opts(N, api.NS_CKPT_STRIDE_HOST, k, lam_coef, 0.0, True, True)
    field = ((w0.size * 8 + 255) // 256) * 256
    # the snapshots before the last segment, whose states stay on the device
    assert S.host_bytes(probe) == ((N - 1) // k - 1) * field
    assert S.host_bytes(S.run_opts(N, api.NS_CKPT_STRIDE, k)) == 0
    # no snapshot in the device arena: smaller than the stride arena once the snapshots
    # outweigh the host tier's device copy of one per pipelined set (40 steps, 9 snapshots)
    assert (S.arena_bytes(S.run_opts(40, api.NS_CKPT_STRIDE_HOST, k, lam_coef)) <
            S.arena_bytes(S.run_opts(40, api.NS_CKPT_STRIDE, k, lam_coef)))
    for pinned in (True, False):
        host = torch.empty(S.host_bytes(probe), dtype=torch.uint8, pin_memory=pinned)
        opts = S.run_opts(N, api.NS_CKPT_STRIDE_HOST, k, lam_coef, 0.0, True, True, host_arena=host)
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
        J = torch.empty(1, dtype=torch.float64, device="cuda")
        lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
        sbar = torch.empty_like(lam0)
        E = torch.zeros((N + 1, 1), dtype=torch.float64, device="cuda")
        st = torch.zeros((N, 1, 2), dtype=torch.float64, device="cuda")
        S.adjoint_run(dev(w0), opts, arena, J, lam0, s=dev(s), sbar=sbar, energy=E, sigma_stats=st)
        torch.cuda.synchronize()
        assert S.last_error() == 0
        for got, want in zip((J, lam0, sbar, E, st), ref):
            assert torch.equal(got, want)
    short = torch.empty(S.host_bytes(probe) - 256, dtype=torch.uint8)
    opts = S.run_opts(N, api.NS_CKPT_STRIDE_HOST, k, lam_coef, host_arena=short)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    with pytest.raises(api.NsError) as e:
        S.adjoint_run(dev(w0), opts, arena, torch.empty(1, dtype=torch.float64, device="cuda"),
                      torch.empty(w0.shape, dtype=torch.float64, device="cuda"))
    assert e.value.code == api.NS_ERR_BUDGET
    opts = S.run_opts(N, api.NS_CKPT_STRIDE_HOST, k, lam_coef)
    with pytest.raises(api.NsError) as e:
        S.adjoint_run(dev(w0), opts, arena, torch.empty(1, dtype=torch.float64, device="cuda"),
                      torch.empty(w0.shape, dtype=torch.float64, device="cuda"))
    assert e.value.code == api.NS_ERR_BUDGET


@pytest.mark.parametrize("prec", [0, 1])
def test_verified_snapshots_keep_the_bits_and_a_corrupted_host_snapshot_is_reported(prec):
    """With verify on, every schedule gives the unverified sweep's bits and a clear error
    word (the verified stride sweeps run their segments in sequence, the unverified ones
    pipelined); a byte flipped in a host-tier snapshot between the forward and the backward
    half (host memory, the caller's arena) is reported as NS_ERR_CORRUPT when the
    snapshot comes back."""
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    N = 13
    S = make_solver(api, w0, P, prec)
    J0, lam0, _, _, _ = _run(api, S, w0, N, api.NS_CKPT_STRIDE, 4)
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam = torch.empty_like(lam0)
    for sched, prm in [(api.NS_CKPT_STRIDE, 4), (api.NS_CKPT_REVOLVE, 3), (api.NS_CKPT_STRIDE_HOST, 4)]:
        host = None
        if sched == api.NS_CKPT_STRIDE_HOST:
            host = torch.zeros(S.host_bytes(S.run_opts(N, sched, prm)), dtype=torch.uint8, pin_memory=True)
        opts = S.run_opts(N, sched, prm, host_arena=host, verify=True)
        if sched == api.NS_CKPT_REVOLVE:
            # the checksums' region; a verified stride sweep (device or host tier) is not
            # pipelined, so it has no second set of replayed states and its arena is the
            # smaller one
            assert S.arena_bytes(opts) > S.arena_bytes(S.run_opts(N, sched, prm, host_arena=host))
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
        S.adjoint_run(dev(w0), opts, arena, J, lam)
        torch.cuda.synchronize()
        assert S.last_error() == 0
        assert torch.equal(J, J0) and torch.equal(lam, lam0)
    # forward half, then a flipped byte in the second host snapshot (step 8), then backward
    host = torch.zeros(S.host_bytes(S.run_opts(N, api.NS_CKPT_STRIDE_HOST, 4)), dtype=torch.uint8,
                       pin_memory=True)
    opts = S.run_opts(N, api.NS_CKPT_STRIDE_HOST, 4, host_arena=host, verify=True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    S.forward_run(dev(w0), opts, arena, J)
    torch.cuda.synchronize()
    slot = host.numel() // 3
    host[slot + 1000] ^= 0x10
    S.backward_run(lam)
    torch.cuda.synchronize()
    assert S.last_error() == api.NS_ERR_CORRUPT
    assert S.last_error() == 0          # the word is cleared by the read


@pytest.mark.parametrize("prec", [0, 1])
def test_disk_snapshots_give_the_stride_bits(prec, tmp_path):
    """NS_CKPT_STRIDE_DISK keeps the every-k-th snapshots in a file (written once in the
    forward pass, read once at replay, through the library's staging buffer): the
    stabilised sweep with a source, energy and sigma_1 series gives the stride schedule's
    bits in the host tier's device memory, and the file is gone when the sweep ends."""
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N, k = 14, 4
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, w0, P, prec)
    ref = _run(api, S, w0, N, 1, k, s, lam_coef=lam_coef, energy=True, sigma=True)
    path = tmp_path / "snapshots.bin"
    opts = S.run_opts(N, api.NS_CKPT_STRIDE_DISK, k, lam_coef, 0.0, True, True, disk_path=str(path), verify=True)
    assert S.host_bytes(opts) == 0
    assert S.arena_bytes(opts) == S.arena_bytes(S.run_opts(N, api.NS_CKPT_STRIDE_HOST, k, lam_coef, 0.0, True, True,
                                                           verify=True))
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    sbar = torch.empty_like(lam0)
    E = torch.zeros((N + 1, 1), dtype=torch.float64, device="cuda")
    st = torch.zeros((N, 1, 2), dtype=torch.float64, device="cuda")
    S.adjoint_run(dev(w0), opts, arena, J, lam0, s=dev(s), sbar=sbar, energy=E, sigma_stats=st)
    torch.cuda.synchronize()
    assert S.last_error() == 0
    for got, want in zip((J, lam0, sbar, E, st), ref):
        assert torch.equal(got, want)
    assert not path.exists()


@pytest.mark.parametrize("prec", [0, 1])
def test_revolve_host_and_disk_tiers_give_the_revolve_bits(prec, tmp_path):
    """NS_CKPT_REVOLVE_HOST / _DISK: the binomial plan with its checkpoints in host memory
    or a file gives NS_CKPT_REVOLVE's bits (stabilised, with a source, energy and sigma_1
    series, verified) in two device states."""
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(33, 10, 3, n=4)[0]
    N, slots = 17, 3
    lam_coef = 0.5 * P.dx[0] ** 2
    S = make_solver(api, w0, P, prec)
    ref = _run(api, S, w0, N, api.NS_CKPT_REVOLVE, slots, s, lam_coef=lam_coef, energy=True, sigma=True)
    field = ((w0.size * 8 + 255) // 256) * 256
    probe = S.run_opts(N, api.NS_CKPT_REVOLVE_HOST, slots, lam_coef, 0.0, True, True)
    assert S.host_bytes(probe) == slots * field
    host = torch.empty(S.host_bytes(probe), dtype=torch.uint8, pin_memory=True)
    for sched, kw in ((api.NS_CKPT_REVOLVE_HOST, {"host_arena": host}),
                      (api.NS_CKPT_REVOLVE_DISK, {"disk_path": str(tmp_path / "rev.bin")})):
        opts = S.run_opts(N, sched, slots, lam_coef, 0.0, True, True, verify=True, **kw)
        assert S.arena_bytes(opts) < S.arena_bytes(S.run_opts(N, api.NS_CKPT_REVOLVE, slots, lam_coef, 0.0, True,
                                                              True, verify=True))
        arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
        J = torch.empty(1, dtype=torch.float64, device="cuda")
        lam0 = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
        sbar = torch.empty_like(lam0)
        E = torch.zeros((N + 1, 1), dtype=torch.float64, device="cuda")
        st = torch.zeros((N, 1, 2), dtype=torch.float64, device="cuda")
        S.adjoint_run(dev(w0), opts, arena, J, lam0, s=dev(s), sbar=sbar, energy=E, sigma_stats=st)
        torch.cuda.synchronize()
        assert S.last_error() == 0
        for got, want in zip((J, lam0, sbar, E, st), ref):
            assert torch.equal(got, want)
    assert not (tmp_path / "rev.bin").exists()


def test_disk_snapshot_errors(tmp_path):
    """A path that cannot be created is NS_ERR_IO before any work is enqueued and a
    missing path NS_ERR_ARG; a byte flipped in the snapshot file between the forward and
    the backward half is NS_ERR_CORRUPT when the snapshot is read back (verify on)."""
    api = _api()
    w0 = synth.isentropic_vortex(33, 10, 3, noise=1e-3, seed=5)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    N, k = 13, 4
    S = make_solver(api, w0, P, 0)
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    lam = torch.empty(w0.shape, dtype=torch.float64, device="cuda")
    bad = S.run_opts(N, api.NS_CKPT_STRIDE_DISK, k, disk_path=str(tmp_path / "missing" / "s.bin"))
    arena = torch.empty(S.arena_bytes(bad), dtype=torch.uint8, device="cuda")
    with pytest.raises(api.NsError) as e:
        S.adjoint_run(dev(w0), bad, arena, J, lam)
    assert e.value.code == api.NS_ERR_IO
    with pytest.raises(api.NsError) as e:
        S.adjoint_run(dev(w0), S.run_opts(N, api.NS_CKPT_STRIDE_DISK, k), arena, J, lam)
    assert e.value.code == api.NS_ERR_ARG
    path = tmp_path / "snapshots.bin"
    opts = S.run_opts(N, api.NS_CKPT_STRIDE_DISK, k, disk_path=str(path), verify=True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    S.forward_run(dev(w0), opts, arena, J)
    torch.cuda.synchronize()
    data = bytearray(path.read_bytes())
    # (N - 1) // k - 1 snapshots (the last segment's first state stays on the device), each
    # at a 256-byte-aligned slot offset
    assert len(data) == ((N - 1) // k - 2) * (((w0.size * 8 + 255) // 256) * 256) + w0.size * 8
    data[len(data) // 3 + 1000] ^= 0x10
    path.write_bytes(bytes(data))
    S.backward_run(lam)
    torch.cuda.synchronize()
    assert S.last_error() == api.NS_ERR_CORRUPT
    assert not path.exists()

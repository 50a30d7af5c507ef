"""GPU choice of the viscosity scaling factor (ns_estimate_lambda) against the oracle's
candidate sweep: per-candidate energy growth, sensitivity change and the chosen index,
in both precision modes, for one box and a batch, plus the argument checks."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_gpu_parity import _api, dev, make_solver
from tests.test_oracle_primal import params_for

pytestmark = pytest.mark.gpu


def _case(nx=20, ny=12, nz=3, seed=3):
    w0 = synth.isentropic_vortex(nx, ny, nz, noise=1e-3, seed=seed)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(nx, ny, nz, n=4)[0]
    return w0, P, s


def _buffers(S, opts):
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device="cuda")
    work = torch.empty(S.estimate_work_bytes(opts), dtype=torch.uint8, device="cuda")
    return arena, work


@pytest.mark.parametrize("prec", [0, 1])
def test_estimate_matches_oracle(prec):
    api = _api()
    w0, P, s = _case()
    N = 8
    lambdas = [0.0, 0.25 * P.dx[0] ** 2, 0.5 * P.dx[0] ** 2, 1.0 * P.dx[0] ** 2, 2.0 * P.dx[0] ** 2]
    chosen_ref, ef_ref, ch_ref, _, _ = O.estimate_lambda(w0, P, N, lambdas, s, efold_tol=1.0, rel_tol=0.1)
    S = make_solver(api, w0, P, prec)
    opts = S.run_opts(N, api.NS_CKPT_STRIDE, 3)
    arena, work = _buffers(S, opts)
    chosen, ef, ch = S.estimate_lambda(dev(w0), opts, lambdas, arena, work, s=dev(s), efold_tol=1.0, rel_tol=0.1)
    assert S.last_error() == 0
    # FP64 mode keeps sigma_1 and nu in FP64 (each sbar to roundoff); mixed mode's FP32
    # products leave about 1e-5 relative in each sbar, and the change is a difference of
    # two sbar fields over the norm of one, which divides that error by the change itself
    # (0.008-0.03 here)
    ef_tol, ch_tol = (1e-9, 1e-10) if prec == 0 else (1e-4, 2e-2)
    np.testing.assert_allclose(ef, ef_ref, rtol=0, atol=ef_tol)
    np.testing.assert_allclose(ch, ch_ref, rtol=ch_tol, atol=1e-12)
    # the choice is unique where no value sits within the tolerance of a threshold
    assert all(abs(c - 0.1) > 4 * ch_tol * max(c, 1e-3) for c in ch_ref)
    assert all(abs(e - 1.0) > 4 * ef_tol for e in ef_ref)
    assert chosen == chosen_ref
    # other thresholds give the oracle's choice on the library's reports (the efolds of
    # this case fall from -0.22 to -0.26 with lambda, the changes rise from 0.008 to 0.03)
    for et, rt in [(1.0, 1e-3), (1.0, 0.05), (-0.235, 0.1), (-0.235, 0.02), (-0.5, 0.1)]:
        assert all(abs(e - et) > 4 * ef_tol for e in ef_ref)
        assert all(abs(c - rt) > 4 * ch_tol * c for c in ch_ref)
        assert api.lambda_select(ef, ch, et, rt) == O.select_lambda(ef_ref, ch_ref, et, rt)
    assert O.select_lambda(ef_ref, ch_ref, -0.235, 0.1) == 3


def test_batch_takes_the_worst_box_and_pools_the_norms():
    api = _api()
    cases = [_case(seed=31), _case(seed=32)]
    w0 = np.stack([c[0] for c in cases])
    P = cases[0][1]
    s = np.stack([c[2] for c in cases])
    N = 6
    lambdas = [0.0, 0.5 * P.dx[0] ** 2, 1.5 * P.dx[0] ** 2]
    refs = [O.estimate_lambda(w0[b], P, N, lambdas, s[b]) for b in range(2)]
    S = make_solver(api, w0[0], P, 0, batch=2)
    opts = S.run_opts(N, api.NS_CKPT_ALL, 0)
    arena, work = _buffers(S, opts)
    chosen, ef, ch = S.estimate_lambda(dev(w0), opts, lambdas, arena, work, s=dev(s))
    ef_ref = [max(refs[0][1][i], refs[1][1][i]) for i in range(len(lambdas))]
    np.testing.assert_allclose(ef, ef_ref, rtol=0, atol=1e-9)
    for i in range(len(lambdas) - 1):
        d2 = sum(np.sum((r[3][i + 1] - r[3][i]) ** 2) for r in refs)
        n2 = sum(np.sum(r[3][i + 1] ** 2) for r in refs)
        assert ch[i] == pytest.approx(math.sqrt(d2) / math.sqrt(n2), rel=1e-10)   # FP64 nu, as above
    assert chosen == O.select_lambda(ef_ref, ch, 1.0, 0.1)


def test_estimate_arguments():
    api = _api()
    w0, P, s = _case(12, 10, 1)
    S = make_solver(api, w0, P, 0)
    opts = S.run_opts(4, api.NS_CKPT_ALL, 0)
    arena, work = _buffers(S, opts)
    wd = dev(w0)
    for bad in ([0.0], [0.0, 0.0], [1e-5, 0.0], [-1e-5, 1e-5]):
        with pytest.raises(api.NsError) as e:
            S.estimate_lambda(wd, opts, bad, arena, work)
        assert e.value.code == api.NS_ERR_ARG
    with pytest.raises(api.NsError) as e:
        S.estimate_lambda(wd, opts, [0.0, 1e-5], arena, work[: work.numel() - 256])
    assert e.value.code == api.NS_ERR_BUDGET
    short = S.run_opts(1, api.NS_CKPT_ALL, 0)
    with pytest.raises(api.NsError) as e:
        S.estimate_lambda(wd, short, [0.0, 1e-5], arena, work)
    assert e.value.code == api.NS_ERR_ARG
    assert S.last_error() == 0

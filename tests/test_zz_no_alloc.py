"""The allocation-free objective entry point (ns_objective_noalloc), called through the C
ABI, gives what the context-based ns_objective gives, on two calls in a row.

Callers that cannot call cudaMalloc (host frameworks that own all device memory, loops
that must not synchronise the device) use this entry point; its reduction scratch is a
fixed device array inside the library, so two calls in a row must not see stale
partial sums from the previous call.  The file name makes pytest collect it last."""
import ctypes
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_06959_gb300 import api, build
    if not os.path.exists(build.OUT):
        build.build()
    lib = api.load_library()
    f = lib.ns_objective_noalloc
    f.argtypes = [ctypes.POINTER(api.NsParams), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return api, lib


def _case(seed, shape=(37, 9, 5), batch=3):
    from paper_1511_06959_gb300 import synth
    ws = np.stack([synth.perturbed_uniform(*shape, seed=seed + i, amp=0.08) for i in range(batch)])
    return ws


def test_noalloc_objective_matches_context_objective_on_two_calls():
    api, lib = _lib()
    nx, ny, nz = 37, 9, 5
    batch = 3
    gamma, mach = 1.4, 0.5
    pt_in = (1 / gamma) * (1 + 0.5 * (gamma - 1) * mach ** 2) ** (gamma / (gamma - 1))
    dx = 1.0 / nx
    S = api.Solver(nx, ny, nz, dx, gamma=gamma, plane_i=(3 * nx) // 4, pt_in=pt_in, batch=batch)
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((5, 17)):
        w = torch.from_numpy(_case(seed, (nx, ny, nz), batch)).cuda()
        J_ref = torch.full((batch,), 0.25, dtype=torch.float64, device="cuda")
        lam_ref = torch.ones_like(w)
        S.objective(w, J_ref, 0.5, lam_ref)
        J = torch.full((batch,), 0.25, dtype=torch.float64, device="cuda")
        lam = torch.ones_like(w)
        rc = lib.ns_objective_noalloc(ctypes.byref(S.params), ctypes.c_void_p(stream.cuda_stream),
                                      ctypes.c_void_p(w.data_ptr()), 0.5, ctypes.c_void_p(J.data_ptr()),
                                      ctypes.c_void_p(lam.data_ptr()))
        assert rc == api.NS_OK, (call, rc)
        torch.cuda.synchronize()
        np.testing.assert_allclose(J.cpu().numpy(), J_ref.cpu().numpy(), rtol=1e-12, atol=0)
        d = (lam - lam_ref).abs().max().item()
        assert d <= 1e-12 * (lam_ref - 1).abs().max().item(), (call, d)


def test_noalloc_objective_rejects_a_batch_beyond_its_scratch():
    api, lib = _lib()
    p = api.NsParams(8, 4, 2, 56, 0.1, 0.1, 0.1, 1.4, 0.0, 0.72, 0.0, 0, 6, 1.0)
    w = torch.zeros(8, dtype=torch.float64, device="cuda")
    J = torch.zeros(56, dtype=torch.float64, device="cuda")
    rc = lib.ns_objective_noalloc(ctypes.byref(p), None, ctypes.c_void_p(w.data_ptr()), 1.0,
                                  ctypes.c_void_p(J.data_ptr()), None)
    assert rc == api.NS_ERR_BUDGET

"""Thin Python binding of the C ABI in include/ns_adjoint.h.

Argument marshalling only: torch CUDA tensors are passed as raw device pointers and
every step runs in the CUDA library.  Importing this module loads
``libns_adjoint.so`` and raises if it has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import weakref

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libns_adjoint.so")

NS_OK = 0
NS_ERR_ARG = -1
NS_ERR_BUDGET = -2
NS_ERR_NONFINITE = -3
NS_ERR_UNSTABLE = -4
NS_ERR_CUDA = -5
NS_ERR_CORRUPT = -6
NS_ERR_BOUNDS = -7
NS_ERR_IO = -8
NS_FP64 = 0
NS_MIXED = 1
NS_RK4 = 0
NS_SSPRK3 = 1
NS_FLUX_CENTRAL = 0
NS_FLUX_ROE = 1
NS_BC_PERIODIC = 0
NS_BC_INOUT = 1
NS_BC_WALLS = 2
NS_BC_INOUT_WALLS = 3
NS_PEAK_FP32 = 0
NS_PEAK_FP32X2 = 1
NS_PEAK_FP64 = 2

EXPORTED = [
    "ns_create", "ns_destroy", "ns_set_stream", "ns_set_dt", "ns_workspace_bytes", "ns_rhs",
    "ns_rhs_tangent", "ns_rhs_transpose", "ns_primal_step", "ns_tangent_step", "ns_adjoint_step",
    "ns_objective", "ns_growth_sigma1", "ns_add_adjoint_viscosity", "ns_apply_adjoint_viscosity",
    "ns_adjoint_energy", "ns_dot", "ns_combine", "ns_max_wave_speed", "ns_last_error",
    "ns_error_string", "ns_plan", "ns_run_arena_bytes", "ns_adjoint_run", "ns_profile_enable",
    "ns_profile_read", "ns_to_float", "ns_forward_run", "ns_backward_run", "ns_scale_boxes",
    "ns_dot_boxes", "ns_mlp_net_bytes", "ns_mlp_set_params", "ns_mlp_get_params", "ns_mlp_get_moment",
    "ns_mlp_features", "ns_mlp_infer", "ns_mlp_train_step", "ns_adjoint_label", "ns_label_target",
    "ns_launch_count", "ns_set_viscosity_split", "ns_set_viscosity_cap", "ns_energy_efolds", "ns_lambda_select",
    "ns_estimate_work_bytes", "ns_estimate_lambda", "ns_run_host_bytes", "ns_measure_fma_peak",
    "ns_sweep_generation", "ns_growth_sigma1_f64", "ns_add_adjoint_viscosity_f64", "ns_adjoint_step_f64",
    "ns_slab_group_create", "ns_slab_group_destroy", "ns_slab_set_exchange", "ns_slab_exchange",
    "ns_slab_primal_step", "ns_slab_adjoint_step", "ns_slab_run_bytes", "ns_slab_adjoint_run", "ns_set_boundaries",
    "ns_adjoint_run_capture", "ns_graph_launch", "ns_graph_kernels", "ns_graph_destroy", "ns_set_pipeline",
]

NS_MLP_PARAMS = 5185

NS_CKPT_ALL = 0
NS_CKPT_STRIDE = 1
NS_CKPT_REVOLVE = 2
NS_CKPT_STRIDE_HOST = 3
NS_CKPT_STRIDE_DISK = 4
NS_CKPT_REVOLVE_HOST = 5
NS_CKPT_REVOLVE_DISK = 6
NS_OP_ADVANCE, NS_OP_STORE, NS_OP_LOAD, NS_OP_ADJOINT, NS_OP_FREE, NS_OP_SOURCE = 1, 2, 3, 4, 5, 6
NS_OP_STORE_HOST, NS_OP_LOAD_HOST, NS_OP_FREE_HOST = 7, 8, 9


class NsParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("batch", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
        ("dt", ctypes.c_double), ("precision", ctypes.c_int), ("plane_i", ctypes.c_int),
        ("pt_in", ctypes.c_double), ("scheme", ctypes.c_int), ("flux", ctypes.c_int),
        ("roe_delta", ctypes.c_double),
    ]


class NsAction(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("a", ctypes.c_int), ("b", ctypes.c_int)]


class NsRunOpts(ctypes.Structure):
    _fields_ = [
        ("nsteps", ctypes.c_int), ("schedule", ctypes.c_int), ("param", ctypes.c_int),
        ("lambda_", ctypes.c_double), ("tau", ctypes.c_double), ("record_energy", ctypes.c_int),
        ("record_sigma", ctypes.c_int), ("mlp", ctypes.c_void_p), ("host_arena", ctypes.c_void_p),
        ("host_bytes", ctypes.c_size_t), ("verify", ctypes.c_int), ("disk_path", ctypes.c_char_p),
    ]


# host ghost-column exchange of a one-slab group (ns_halo_exchange_fn)
HALO_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)


class NsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib().ns_error_string(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


_LIB = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library and declare its signatures."""
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library not built: {path} is missing (run paper_1511_06959_gb300.build)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    S = ctypes.c_size_t
    sig = {
        "ns_create": ([ctypes.POINTER(NsParams), P, ctypes.POINTER(P)], I),
        "ns_destroy": ([P], None),
        "ns_set_stream": ([P, P], I),
        "ns_set_dt": ([P, D], I),
        "ns_workspace_bytes": ([P], S),
        "ns_rhs": ([P, P, P, P], I),
        "ns_rhs_tangent": ([P, P, P, P], I),
        "ns_rhs_transpose": ([P, P, P, P, P], I),
        "ns_primal_step": ([P, P, P, P], I),
        "ns_tangent_step": ([P, P, P, P, P, P], I),
        "ns_adjoint_step": ([P, P, P, P, P, P, P], I),
        "ns_objective": ([P, P, D, P, P], I),
        "ns_growth_sigma1": ([P, P, P, P], I),
        "ns_add_adjoint_viscosity": ([P, P, D, D, P], I),
        "ns_apply_adjoint_viscosity": ([P, P, P, P], I),
        "ns_adjoint_energy": ([P, P, P, P], I),
        "ns_dot": ([P, P, P, I, S, P], I),
        "ns_combine": ([P, P, P, I, S, P], I),
        "ns_max_wave_speed": ([P, P, P], I),
        "ns_to_float": ([P, P, P, S], I),
        "ns_forward_run": ([P, P, P, ctypes.POINTER(NsRunOpts), P, S, P], I),
        "ns_backward_run": ([P, P, P, P, P], I),
        "ns_scale_boxes": ([P, P, P], I),
        "ns_dot_boxes": ([P, P, I, P, I, P], I),
        "ns_mlp_net_bytes": ([], S),
        "ns_mlp_set_params": ([P, P, P], I),
        "ns_mlp_get_params": ([P, P, P], I),
        "ns_mlp_get_moment": ([P, P, I, P], I),
        "ns_mlp_features": ([P, P, P], I),
        "ns_mlp_infer": ([P, P, P, P, D, P], I),
        "ns_mlp_train_step": ([P, P, P, P, P, I, I, D, P], I),
        "ns_adjoint_label": ([P, P, P, P], I),
        "ns_label_target": ([P, P, P, D, P], I),
        "ns_last_error": ([P], I),
        "ns_error_string": ([I], ctypes.c_char_p),
        "ns_launch_count": ([], ctypes.c_ulonglong),
        "ns_measure_fma_peak": ([I, ctypes.POINTER(D)], I),
        "ns_sweep_generation": ([P], ctypes.c_longlong),
        "ns_growth_sigma1_f64": ([P, P, P, P], I),
        "ns_add_adjoint_viscosity_f64": ([P, P, D, D, P], I),
        "ns_adjoint_step_f64": ([P, P, P, P, P, P, P], I),
        "ns_set_boundaries": ([P, I, ctypes.POINTER(D), ctypes.POINTER(D)], I),
        "ns_slab_group_create": ([ctypes.POINTER(P), I, ctypes.POINTER(P)], I),
        "ns_slab_group_destroy": ([P], None),
        "ns_slab_set_exchange": ([P, HALO_FN, P], I),
        "ns_slab_exchange": ([P, ctypes.POINTER(P), I, I], I),
        "ns_slab_primal_step": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)], I),
        "ns_slab_run_bytes": ([P, ctypes.POINTER(NsRunOpts), ctypes.POINTER(ctypes.c_size_t)], I),
        "ns_slab_adjoint_run": ([P, I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(NsRunOpts),
                                 ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t), P, ctypes.POINTER(P)], I),
        "ns_slab_adjoint_step": ([P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                  ctypes.POINTER(P)], I),
        "ns_set_viscosity_split": ([P, ctypes.POINTER(ctypes.c_double)], I),
        "ns_set_viscosity_cap": ([P, I], I),
        "ns_plan": ([I, I, I, P, I, ctypes.POINTER(I), ctypes.POINTER(I),
                     ctypes.POINTER(ctypes.c_longlong)], I),
        "ns_run_arena_bytes": ([P, ctypes.POINTER(NsRunOpts)], S),
        "ns_run_host_bytes": ([P, ctypes.POINTER(NsRunOpts)], S),
        "ns_adjoint_run": ([P, P, P, ctypes.POINTER(NsRunOpts), P, S, P, P, P, P, P], I),
        "ns_adjoint_run_capture": ([P, P, P, ctypes.POINTER(NsRunOpts), P, S, P, P, P, P, P,
                                    ctypes.POINTER(ctypes.c_void_p)], I),
        "ns_graph_launch": ([P], I),
        "ns_set_pipeline": ([P, I], I),
        "ns_graph_kernels": ([P], ctypes.c_longlong),
        "ns_graph_destroy": ([P], None),
        "ns_profile_enable": ([P, I], I),
        "ns_profile_read": ([P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)], I),
        "ns_energy_efolds": ([ctypes.POINTER(D), I, I, ctypes.POINTER(D)], I),
        "ns_lambda_select": ([I, ctypes.POINTER(D), ctypes.POINTER(D), D, D], I),
        "ns_estimate_work_bytes": ([P, ctypes.POINTER(NsRunOpts)], S),
        "ns_estimate_lambda": ([P, P, P, ctypes.POINTER(NsRunOpts), ctypes.POINTER(D), I, D, D, P, S, P, S,
                                ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I)], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


def _lib() -> ctypes.CDLL:
    """The library, loaded on first use: libns_adjoint.so next to this file, or the
    build named by the environment variable NS_ADJOINT_LIB (such as the bounds-checking
    build, paper_1511_06959_gb300.build.build(debug=True))."""
    global _LIB
    if _LIB is None:
        _LIB = load_library(os.environ.get("NS_ADJOINT_LIB") or LIB_PATH)
    return _LIB


def _doubles(values):
    values = [float(v) for v in values]
    return (ctypes.c_double * max(len(values), 1))(*values)


def energy_efolds(E, nsteps: int, batch: int = 1):
    """Energy growth over the second half of the backward sweep, in e-folds, per box
    (host computation); E is a flat or [nsteps+1][batch] sequence of floats."""
    flat = [float(v) for row in E for v in (row if hasattr(row, "__len__") else [row])]
    out = (ctypes.c_double * batch)()
    _check(_lib().ns_energy_efolds(_doubles(flat), nsteps, batch, out), "ns_energy_efolds")
    return list(out)


def lambda_select(efolds, change, efold_tol: float, rel_tol: float) -> int:
    """Index of the smallest damped candidate on the sensitivity plateau, or -1."""
    return int(_lib().ns_lambda_select(len(efolds), _doubles(efolds), _doubles(change), efold_tol, rel_tol))


def plan(nsteps: int, schedule: int, param: int = 0):
    """Checkpoint plan (host computation): (actions as (op, a, b) tuples, slots, advances)."""
    lib = _lib()
    n = ctypes.c_int()
    slots = ctypes.c_int()
    adv = ctypes.c_longlong()
    _check(lib.ns_plan(nsteps, schedule, param, None, 0, ctypes.byref(n), ctypes.byref(slots),
                       ctypes.byref(adv)), "ns_plan")
    arr = (NsAction * max(n.value, 1))()
    _check(lib.ns_plan(nsteps, schedule, param, arr, n.value, ctypes.byref(n), ctypes.byref(slots),
                       ctypes.byref(adv)), "ns_plan")
    return [(a.op, a.a, a.b) for a in arr[: n.value]], slots.value, adv.value


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _sized(t, dtype, n, what):
    """_ptr of a tensor that must hold at least n elements (the library writes or reads n
    of them through the raw pointer), or None for None."""
    if t is None:
        return None
    if t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the call uses {n}")
    return _ptr(t, dtype)


def _host_ptr(t):
    """Address of a contiguous CPU tensor (host memory for the library), or None."""
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("expected a CPU tensor (host memory)")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(code: int, where: str):
    if code != NS_OK:
        raise NsError(code, where)


class Solver:
    """One context of the C library: a periodic box (or a batch of boxes) with fixed
    physical parameters, precision and time step."""

    def __init__(self, nx, ny, nz, dx, gamma=1.4, mu=0.0, Pr=0.72, dt=0.0, precision=NS_FP64,
                 plane_i=0, pt_in=1.0, batch=1, stream=None, scheme=NS_RK4, flux=NS_FLUX_CENTRAL,
                 roe_delta=0.1):
        self.lib = _lib()
        d = dx if isinstance(dx, (tuple, list)) else (dx, dx, dx)
        self.params = NsParams(nx, ny, nz, batch, d[0], d[1], d[2], gamma, mu, Pr, dt,
                               precision, plane_i, pt_in, scheme, flux, roe_delta)
        self.nstages = 3 if scheme == NS_SSPRK3 else 4
        self.shape = (batch, 5, nz, ny, nx)
        self.cells = nx * ny * nz
        self.batch = batch
        self._ctx = ctypes.c_void_p()
        self._graphs = []   # weak references to this context's captured sweeps
        st = stream if stream is not None else torch.cuda.current_stream()
        _check(self.lib.ns_create(ctypes.byref(self.params), ctypes.c_void_p(st.cuda_stream),
                                  ctypes.byref(self._ctx)), "ns_create")

    # size-checked device pointers: a 5-component field, a scalar field, one value per box
    def _F(self, t, dtype=torch.float64):
        return _sized(t, dtype, self.batch * 5 * self.cells, "field")

    def _S(self, t, dtype=torch.float32):
        return _sized(t, dtype, self.batch * self.cells, "scalar field")

    def _B(self, t, per_box=1):
        return _sized(t, torch.float64, self.batch * per_box, "per-box array")

    def close(self):
        # a captured sweep refers to the context: released first
        for ref in getattr(self, "_graphs", []):
            g = ref()
            if g is not None:
                g.close()
        if self._ctx:
            self.lib.ns_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dt(self):
        return self.params.dt

    def set_dt(self, dt):
        self.params.dt = dt
        _check(self.lib.ns_set_dt(self._ctx, dt), "ns_set_dt")

    def set_stream(self, stream):
        _check(self.lib.ns_set_stream(self._ctx, ctypes.c_void_p(stream.cuda_stream)), "ns_set_stream")

    def workspace_bytes(self):
        return int(self.lib.ns_workspace_bytes(self._ctx))

    # --- field operations -------------------------------------------------------
    def rhs(self, w, R, s=None):
        _check(self.lib.ns_rhs(self._ctx, self._F(w), self._F(s),
                               self._F(R)), "ns_rhs")

    def rhs_tangent(self, w, wd, Rd):
        _check(self.lib.ns_rhs_tangent(self._ctx, self._F(w), self._F(wd),
                                       self._F(Rd)), "ns_rhs_tangent")

    def rhs_transpose(self, w, a, out, nu=None):
        _check(self.lib.ns_rhs_transpose(self._ctx, self._F(w), self._F(a),
                                         self._S(nu), self._F(out)),
               "ns_rhs_transpose")

    def primal_step(self, w_in, w_out, s=None):
        _check(self.lib.ns_primal_step(self._ctx, self._F(w_in), self._F(s),
                                       self._F(w_out)), "ns_primal_step")

    def tangent_step(self, w, wd_in, wd_out, s=None, sd=None):
        _check(self.lib.ns_tangent_step(self._ctx, self._F(w), self._F(s),
                                        self._F(wd_in), self._F(sd),
                                        self._F(wd_out)), "ns_tangent_step")

    def adjoint_step(self, w_n, lam_np1, lam_n, s=None, nu=None, sbar=None):
        """A float64 nu selects ns_adjoint_step_f64 (FP64 contexts), a float32 one (or
        None) ns_adjoint_step."""
        if nu is not None and nu.dtype == torch.float64:
            _check(self.lib.ns_adjoint_step_f64(self._ctx, self._F(w_n), self._F(s),
                                                self._F(lam_np1), self._S(nu, torch.float64),
                                                self._F(lam_n), self._F(sbar)),
                   "ns_adjoint_step_f64")
            return
        _check(self.lib.ns_adjoint_step(self._ctx, self._F(w_n), self._F(s),
                                        self._F(lam_np1), self._S(nu),
                                        self._F(lam_n), self._F(sbar)),
               "ns_adjoint_step")

    def objective(self, w, J_acc, weight=1.0, lam=None):
        _check(self.lib.ns_objective(self._ctx, self._F(w), float(weight),
                                     self._B(J_acc), self._F(lam)),
               "ns_objective")

    def growth_sigma1(self, w, sigma1, stats=None):
        """A float64 sigma1 selects ns_growth_sigma1_f64 (FP64 contexts)."""
        if sigma1.dtype == torch.float64:
            _check(self.lib.ns_growth_sigma1_f64(self._ctx, self._F(w), self._S(sigma1, torch.float64),
                                                 self._B(stats, 2)), "ns_growth_sigma1_f64")
            return
        _check(self.lib.ns_growth_sigma1(self._ctx, self._F(w), self._S(sigma1),
                                         self._B(stats, 2)), "ns_growth_sigma1")

    def add_adjoint_viscosity(self, sigma1, lam_coef, nu, tau=0.0):
        """A float64 sigma1 selects ns_add_adjoint_viscosity_f64 (nu float64 too)."""
        if sigma1.dtype == torch.float64:
            _check(self.lib.ns_add_adjoint_viscosity_f64(self._ctx, self._S(sigma1, torch.float64), float(lam_coef),
                                                         float(tau), self._S(nu, torch.float64)),
                   "ns_add_adjoint_viscosity_f64")
            return
        _check(self.lib.ns_add_adjoint_viscosity(self._ctx, self._S(sigma1), float(lam_coef),
                                                 float(tau), self._S(nu)),
               "ns_add_adjoint_viscosity")

    def apply_adjoint_viscosity(self, nu, a, out):
        _check(self.lib.ns_apply_adjoint_viscosity(self._ctx, self._S(nu),
                                                   self._F(a), self._F(out)),
               "ns_apply_adjoint_viscosity")

    def adjoint_energy(self, w, lam, E):
        _check(self.lib.ns_adjoint_energy(self._ctx, self._F(w), self._F(lam),
                                          self._B(E)), "ns_adjoint_energy")

    def dot(self, a, phi, out):
        nphi = phi.shape[0]
        n = a.numel()
        if phi.numel() != nphi * n:
            raise ValueError("phi must be [nphi, a.numel()]")
        _check(self.lib.ns_dot(self._ctx, _ptr(a, torch.float64), _ptr(phi, torch.float64), nphi, n,
                               _ptr(out, torch.float64)), "ns_dot")

    def combine(self, theta, phi, s):
        nphi = phi.shape[0]
        n = s.numel()
        _check(self.lib.ns_combine(self._ctx, _ptr(theta, torch.float64), _ptr(phi, torch.float64), nphi,
                                   n, _ptr(s, torch.float64)), "ns_combine")

    def to_float(self, x, out):
        _check(self.lib.ns_to_float(self._ctx, _ptr(x, torch.float64), _ptr(out, torch.float32), x.numel()),
               "ns_to_float")

    def max_wave_speed(self, w, out):
        _check(self.lib.ns_max_wave_speed(self._ctx, self._F(w), _ptr(out, torch.float64)),
               "ns_max_wave_speed")

    def set_boundaries(self, bc: int, far=None, wall_e=None):
        """Characteristic inflow/outflow in x and/or isothermal walls in y
        (ns_set_boundaries); far = (rho, u1, u2, u3, p), wall_e = (bottom, top)."""
        _check(self.lib.ns_set_boundaries(self._ctx, int(bc), None if far is None else _doubles(far),
                                          None if wall_e is None else _doubles(wall_e)), "ns_set_boundaries")

    def set_viscosity_split(self, f_rho: float, f_mom: float, f_en: float):
        arr = (ctypes.c_double * 3)(f_rho, f_mom, f_en)
        _check(self.lib.ns_set_viscosity_split(self._ctx, arr), "ns_set_viscosity_split")

    def set_viscosity_cap(self, cap: bool):
        """Hold the added viscosity at the explicit stability limit instead of flagging it
        (ns_set_viscosity_cap)."""
        _check(self.lib.ns_set_viscosity_cap(self._ctx, int(bool(cap))), "ns_set_viscosity_cap")

    def set_pipeline(self, on: bool):
        """Pipelined stride sweeps (the next segment replayed on a second stream while the
        current one is reversed) on or off (ns_set_pipeline); arena_bytes follows."""
        _check(self.lib.ns_set_pipeline(self._ctx, int(bool(on))), "ns_set_pipeline")

    def last_error(self) -> int:
        return int(self.lib.ns_last_error(self._ctx))

    # --- checkpointed sweep ----------------------------------------------------------
    def run_opts(self, nsteps, schedule=NS_CKPT_ALL, param=0, lam_coef=0.0, tau=0.0,
                 record_energy=False, record_sigma=False, mlp=None, host_arena=None, verify=False,
                 disk_path=None):
        """Sweep options; mlp: a network blob (uint8 CUDA tensor) selecting the learned
        closure, with lam_coef then its global factor kappa; host_arena: a uint8 CPU
        tensor (pinned for asynchronous copies) holding the snapshots of an
        NS_CKPT_STRIDE_HOST sweep (the options keep a reference to it); verify: checksum
        every snapshot when stored and check it when loaded (NS_ERR_CORRUPT); disk_path: the
        snapshot file of an NS_CKPT_STRIDE_DISK sweep."""
        o = NsRunOpts(nsteps, schedule, param, lam_coef, tau, int(record_energy), int(record_sigma),
                      None if mlp is None else ctypes.c_void_p(mlp.data_ptr()),
                      _host_ptr(host_arena),
                      0 if host_arena is None else host_arena.numel() * host_arena.element_size(),
                      int(verify), None if disk_path is None else os.fsencode(disk_path))
        o._host_arena = host_arena
        return o

    def arena_bytes(self, opts) -> int:
        return int(self.lib.ns_run_arena_bytes(self._ctx, ctypes.byref(opts)))

    def host_bytes(self, opts) -> int:
        """Host bytes of an NS_CKPT_STRIDE_HOST or NS_CKPT_REVOLVE_HOST sweep's snapshot
        arena (0 otherwise)."""
        return int(self.lib.ns_run_host_bytes(self._ctx, ctypes.byref(opts)))

    def adjoint_run(self, w0, opts, arena, Jbar, lam0, s=None, sbar=None, energy=None,
                    sigma_stats=None):
        """Forward + checkpointed backward sweep; arena is a uint8 CUDA tensor of at least
        arena_bytes(opts) bytes."""
        N = opts.nsteps
        _check(self.lib.ns_adjoint_run(self._ctx, self._F(w0), self._F(s),
                                       ctypes.byref(opts), _ptr(arena), arena.numel() * arena.element_size(),
                                       self._B(Jbar), self._F(lam0), self._F(sbar), self._B(energy, N + 1),
                                       self._B(sigma_stats, 2 * N)), "ns_adjoint_run")

    def adjoint_run_capture(self, w0, opts, arena, Jbar, lam0, s=None, sbar=None, energy=None,
                            sigma_stats=None):
        """adjoint_run recorded as one CUDA graph (nothing runs yet); returns a SweepGraph
        whose launch() replays the whole sweep on the solver's stream."""
        N = opts.nsteps
        g = ctypes.c_void_p()
        _check(self.lib.ns_adjoint_run_capture(self._ctx, self._F(w0), self._F(s),
                                               ctypes.byref(opts), _ptr(arena),
                                               arena.numel() * arena.element_size(), self._B(Jbar),
                                               self._F(lam0), self._F(sbar), self._B(energy, N + 1),
                                               self._B(sigma_stats, 2 * N), ctypes.byref(g)),
               "ns_adjoint_run_capture")
        return SweepGraph(self, g)

    def estimate_work_bytes(self, opts) -> int:
        return int(self.lib.ns_estimate_work_bytes(self._ctx, ctypes.byref(opts)))

    def estimate_lambda(self, w0, opts, lambdas, arena, work, s=None, efold_tol=1.0, rel_tol=0.1):
        """One stabilised sweep per candidate factor (ascending); returns (chosen index or
        -1, energy growth in e-folds per candidate, relative sensitivity change per
        consecutive pair).  arena: as for adjoint_run; work: a uint8 CUDA tensor of at
        least estimate_work_bytes(opts) bytes."""
        n = len(lambdas)
        ef = (ctypes.c_double * n)()
        ch = (ctypes.c_double * max(n - 1, 1))()
        chosen = ctypes.c_int(-1)
        _check(self.lib.ns_estimate_lambda(self._ctx, _ptr(w0, torch.float64), _ptr(s, torch.float64),
                                           ctypes.byref(opts), _doubles(lambdas), n, efold_tol, rel_tol,
                                           _ptr(arena), arena.numel() * arena.element_size(), _ptr(work),
                                           work.numel() * work.element_size(), ef, ch, ctypes.byref(chosen)),
               "ns_estimate_lambda")
        return chosen.value, list(ef), list(ch)[: max(n - 1, 0)]

    def forward_run(self, w0, opts, arena, Jbar, s=None):
        """Forward half of the sweep (keeps the checkpoints in arena, accumulates Jbar)."""
        _check(self.lib.ns_forward_run(self._ctx, self._F(w0), self._F(s),
                                       ctypes.byref(opts), _ptr(arena), arena.numel() * arena.element_size(),
                                       self._B(Jbar)), "ns_forward_run")
        self._fwd_steps = opts.nsteps

    def sweep_generation(self) -> int:
        """Number of the forward sweep awaiting its backward, 0 if none (ns_sweep_generation)."""
        return int(self.lib.ns_sweep_generation(self._ctx))

    def backward_run(self, lam0, sbar=None, energy=None, sigma_stats=None):
        """Reverse half of the sweep with a unit seed on each box's Jbar."""
        N = getattr(self, "_fwd_steps", 0)
        _check(self.lib.ns_backward_run(self._ctx, self._F(lam0), self._F(sbar),
                                        self._B(energy, N + 1), self._B(sigma_stats, 2 * N)),
               "ns_backward_run")

    def scale_boxes(self, seed, field):
        _check(self.lib.ns_scale_boxes(self._ctx, _ptr(seed, torch.float64), _ptr(field, torch.float64)),
               "ns_scale_boxes")

    def dot_boxes(self, field, comp, phi, out):
        _check(self.lib.ns_dot_boxes(self._ctx, _ptr(field, torch.float64), int(comp),
                                     _ptr(phi, torch.float64), phi.shape[0], _ptr(out, torch.float64)),
               "ns_dot_boxes")

    # --- learned closure -------------------------------------------------------------
    def mlp_set_params(self, net, params):
        _check(self.lib.ns_mlp_set_params(self._ctx, _ptr(net), _ptr(params, torch.float32)), "ns_mlp_set_params")

    def mlp_get_params(self, net, out):
        _check(self.lib.ns_mlp_get_params(self._ctx, _ptr(net), _ptr(out, torch.float32)), "ns_mlp_get_params")

    def mlp_get_moment(self, net, which, out):
        _check(self.lib.ns_mlp_get_moment(self._ctx, _ptr(net), int(which), _ptr(out, torch.float32)),
               "ns_mlp_get_moment")

    def mlp_features(self, w, feat):
        _check(self.lib.ns_mlp_features(self._ctx, self._F(w), _sized(feat, torch.float32, 16 * self.batch * self.cells, "features")),
               "ns_mlp_features")

    def mlp_infer(self, net, feat, sigma1, kappa, nu):
        _check(self.lib.ns_mlp_infer(self._ctx, _ptr(net), _ptr(feat, torch.float32), _ptr(sigma1, torch.float32),
                                     float(kappa), _ptr(nu, torch.float32)), "ns_mlp_infer")

    def mlp_train_step(self, net, feat, target, idx, step, lr, loss=None):
        _check(self.lib.ns_mlp_train_step(self._ctx, _ptr(net), _ptr(feat, torch.float32),
                                          _ptr(target, torch.float32), _ptr(idx, torch.int32), idx.numel(),
                                          int(step), float(lr), _ptr(loss, torch.float32)), "ns_mlp_train_step")

    def adjoint_label(self, w, lam, acc):
        _check(self.lib.ns_adjoint_label(self._ctx, self._F(w), self._F(lam), self._S(acc)), "ns_adjoint_label")

    def label_target(self, acc, sigma1, t_max, target):
        _check(self.lib.ns_label_target(self._ctx, _ptr(acc, torch.float32), _ptr(sigma1, torch.float32),
                                        float(t_max), _ptr(target, torch.float32)), "ns_label_target")

    def profile_enable(self, on=True):
        _check(self.lib.ns_profile_enable(self._ctx, int(on)), "ns_profile_enable")

    def profile_read(self):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(self.lib.ns_profile_read(self._ctx, ctypes.byref(ms), ctypes.byref(n)), "ns_profile_read")
        return ms.value, n.value


def launch_count() -> int:
    """Kernels this library has launched in this process (ns_launch_count)."""
    return int(_lib().ns_launch_count())


def mlp_net_bytes() -> int:
    return int(_lib().ns_mlp_net_bytes())


def measure_fma_peak(kind: int) -> float:
    """Measured multiply-add rate of the current device in flop/s (ns_measure_fma_peak);
    kind is NS_PEAK_FP32, NS_PEAK_FP32X2 or NS_PEAK_FP64."""
    out = ctypes.c_double()
    _check(_lib().ns_measure_fma_peak(int(kind), ctypes.byref(out)), "ns_measure_fma_peak")
    return out.value


class SweepGraph:
    """One sweep captured as a CUDA graph (Solver.adjoint_run_capture).  launch() replays
    the whole sweep on the solver's stream, reading w0 and s as they are then and
    overwriting the outputs given at capture; kernels is the number of this library's
    kernel launches in one replay."""

    def __init__(self, solver, handle):
        self.solver = solver
        self.lib = solver.lib
        self._g = handle
        solver._graphs.append(weakref.ref(self))

    @property
    def kernels(self) -> int:
        return int(self.lib.ns_graph_kernels(self._g))

    def launch(self):
        _check(self.lib.ns_graph_launch(self._g), "ns_graph_launch")

    def close(self):
        if self._g:
            self.lib.ns_graph_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(tensors, dtype, sizes=None):
    """A host array of device pointers (one per slab), or None; sizes: the elements the
    call uses in each."""
    if tensors is None:
        return None
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _ptr(t, dtype) if sizes is None else _sized(t, dtype, sizes[i], "slab field")
    return arr


class SlabGroup:
    """x-slabs of one box, each a Solver over its padded slab (one ghost column per
    side), stepped together with their ghost columns exchanged after every stage
    (ns_slab_*)."""

    def __init__(self, solvers, exchange=None):
        self.lib = _lib()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s._ctx for s in self.solvers])
        g = ctypes.c_void_p()
        _check(self.lib.ns_slab_group_create(arr, len(self.solvers), ctypes.byref(g)), "ns_slab_group_create")
        self._g = g
        self._fn = None
        if exchange is not None:
            # exchange(field_tensor_view_args) is called as exchange(ptr, elem_bytes, ncomp)
            self._fn = HALO_FN(lambda user, field, eb, nc: int(exchange(field, eb, nc) or 0))
            _check(self.lib.ns_slab_set_exchange(self._g, self._fn, None), "ns_slab_set_exchange")

    def close(self):
        if getattr(self, "_g", None):
            self.lib.ns_slab_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sizes(self, ncomp):
        return [s.batch * ncomp * s.cells for s in self.solvers]

    def exchange(self, fields, ncomp):
        if len(fields) != len(self.solvers):
            raise ValueError("one field per slab")
        eb = fields[0].element_size()
        _check(self.lib.ns_slab_exchange(self._g, _ptr_array(fields, fields[0].dtype, self._sizes(ncomp)), eb,
                                         ncomp), "ns_slab_exchange")

    def primal_step(self, w, wo, s=None):
        f = self._sizes(5)
        _check(self.lib.ns_slab_primal_step(self._g, _ptr_array(w, torch.float64, f),
                                            _ptr_array(s, torch.float64, f), _ptr_array(wo, torch.float64, f)),
               "ns_slab_primal_step")

    def adjoint_step(self, w, lam, lo, s=None, nu=None):
        f = self._sizes(5)
        _check(self.lib.ns_slab_adjoint_step(self._g, _ptr_array(w, torch.float64, f),
                                             _ptr_array(s, torch.float64, f), _ptr_array(lam, torch.float64, f),
                                             _ptr_array(nu, torch.float32, self._sizes(1)),
                                             _ptr_array(lo, torch.float64, f)), "ns_slab_adjoint_step")

    def run_bytes(self, opts):
        """Workspace bytes of adjoint_run for each slab (ns_slab_run_bytes)."""
        out = (ctypes.c_size_t * len(self.solvers))()
        _check(self.lib.ns_slab_run_bytes(self._g, ctypes.byref(opts), out), "ns_slab_run_bytes")
        return list(out)

    def adjoint_run(self, own, w0, opts, work, Jbar, lam0, s=None):
        """The checkpointed sweep on the group (ns_slab_adjoint_run): slab `own` holds the
        objective plane; work: one uint8 CUDA tensor per slab of at least run_bytes."""
        f = self._sizes(5)
        if len(work) != len(self.solvers):
            raise ValueError("one workspace per slab")
        warr = (ctypes.c_void_p * len(work))(*[_ptr(t) for t in work])
        wb = (ctypes.c_size_t * len(work))(*[t.numel() * t.element_size() for t in work])
        _check(self.lib.ns_slab_adjoint_run(self._g, int(own), _ptr_array(w0, torch.float64, f),
                                            _ptr_array(s, torch.float64, f), ctypes.byref(opts), warr, wb,
                                            _sized(Jbar, torch.float64, self.solvers[own].batch, "Jbar"),
                                            _ptr_array(lam0, torch.float64, f)), "ns_slab_adjoint_run")

#!/usr/bin/env python
"""Benchmark of the checkpointed unsteady discrete adjoint on one GB300 per rank.

One step = the whole hot path over one synthetic box: the RK4 primal forward pass
with the pressure-loss objective, then the backward sweep that replays each
checkpoint segment, evaluates sigma_1 and the added adjoint viscosity, applies the four
transposed RK4 stages, adds the objective source and records the adjoint energy.
The metric is adjoint cell-steps/s (cells x RK4 steps reversed, per second).  Each step
is one launch of the sweep captured once as a CUDA graph (all of its kernels run again
every step); --no-graph times the sweep call itself.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload box128]
                  [--precision mixed|fp64] [--impl ours|reference] [--no-graph]

Under torchrun each rank runs its own independent box (weak scaling, no data-path
collective); rank 0 prints one JSON line.  --impl reference times the FP64 CPU
oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1511_06959_gb300 import config as C  # noqa: E402

METRIC = "adjoint cell-steps/s and % HBM roofline, mixed+checkpointed vs FP64 at stated grad err"
UNIT = "adjoint cell-steps/s"

# Algorithmic bytes per adjoint cell-step, the minimum the method must move: read w^n,
# read lam^{n+1}, write lam^n, 5 FP64 values each (120 B, the same in mixed precision,
# whose state and adjoint stay FP64).  One adjoint-stage launch does 1/stages of a step.
# The checkpointed sweep adds the replay's read and write of the state: about 200 B per
# adjoint cell-step in all.
ADJ_STEP_BYTES = 120.0
SWEEP_BYTES = 200.0
# operand bytes per cell that the adjoint-stage kernel itself reads and writes, averaged
# over the four RK4 stages (float mirrors, kept stage states, seeds and sums in mixed
# precision; nu present, no source seed): a design figure, not the algorithmic minimum
ADJ_STAGE_OPERAND_BYTES = {"mixed": (124 + 184 + 184 + 144) / 4.0, "fp64": (164 + 244 + 244 + 164) / 4.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="box128", choices=sorted(C.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nu-split", default="1,1,1",
                    help="added-viscosity factors for the rho, rho u, rho E adjoints")
    ap.add_argument("--closure", action="store_true",
                    help="the learned viscosity closure (an MLP network, kappa = 0.5) inside the sweep "
                         "instead of the sigma_1 rule")
    ap.add_argument("--flux", default="central", choices=["central", "roe"],
                    help="convective face flux (the workload's is central; roe adds the paper's "
                         "Roe dissipation)")
    ap.add_argument("--scheme", default="rk4", choices=["rk4", "ssprk3"],
                    help="time integrator (the workload's is RK4; ssprk3 is the paper's own)")
    ap.add_argument("--host-snapshots", action="store_true",
                    help="keep a stride schedule's snapshots in page-locked host memory")
    ap.add_argument("--disk-snapshots", default=None, metavar="PATH",
                    help="keep a stride schedule's snapshots in the file PATH (removed after each sweep)")
    ap.add_argument("--no-graph", action="store_true",
                    help="time the sweep call itself instead of its captured CUDA graph")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nsteps", type=int, default=0,
                    help="override the workload's RK4 step count (profiling runs)")
    return ap.parse_args()


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------------
# CPU oracle: one checkpointed adjoint step of the workload on the host cores
# ----------------------------------------------------------------------------------
def oracle_unit(w, P, lam_tilde, dx0):
    """Forward step + replay step + stabilised adjoint step (sigma_1, nu, objective source,
    adjoint energy) of the full box: the work the GPU sweep does per reversed step."""
    from oracle import ns_oracle as O
    w1, _ = O.step(w, P)
    O.objective(w1, P)
    w1, _ = O.step(w, P)
    lam = O.objective_grad(w1, P)
    nu = lam_tilde * dx0 ** 2 * O.sigma1_field(w, P)
    lam, _ = O.adjoint_step(w, lam, P, None, nu)
    lam = lam + O.objective_grad(w, P)
    O.adjoint_energy(w, lam, P)


def oracle_setup(wl, scheme="rk4", flux="central"):
    from oracle import ns_oracle as O
    w = wl.initial_state()
    P = O.Params(gamma=wl.gamma, mu=wl.mu, Pr=wl.Pr, dx=wl.dx, plane_i=wl.plane_i, pt_in=wl.pt_in,
                 scheme=scheme, flux=flux)
    P.dt = C.cfl_dt(wl, O.max_wave_speed(w, P))
    return w, P


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, wl):
    ws, rank, _ = dist_init()
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    w, P = oracle_setup(wl, args.scheme, args.flux)
    for _ in range(min(args.warmup, 1)):
        oracle_unit(w, P, wl.lam_tilde, wl.dx[0])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_unit(w, P, wl.lam_tilde, wl.dx[0])
    t = time.perf_counter() - t0
    v = args.steps * wl.cells * wl.batch / t
    sample = (f"{args.steps} x one checkpointed adjoint step (forward + replay + stabilised "
              f"adjoint + source + energy) of the full {wl.nx}x{wl.ny}x{wl.nz} box")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": min(args.warmup, 1), "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": C.describe(wl, args.scheme, args.flux), "name": wl.name,
                                        "scheme": args.scheme, "flux": args.flux},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus_id = bus_id
        self.proc = None
        import tempfile
        out = os.environ.get("NS_RESULTS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.bus_id:
                cmd.insert(1, f"--id={self.bus_id}")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), float(p[3]), p[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        pmax = max(r[2] for r in rows)
        load = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": pmax}


def max_over_ranks(ms, t_e2e, ws, device):
    """The slowest rank's step time and end-to-end time (every rank gets them)."""
    if ws <= 1:
        return ms, t_e2e
    import torch
    tt = torch.tensor([ms, t_e2e], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return tt[0].item(), tt[1].item()


def whole_job_rates(ws, cell_steps, ms, t_e2e):
    """Adjoint cell-steps/s of the whole job: every rank reverses its own box (weak
    scaling, no data-path collective), so the job's work is ws boxes in the slowest
    rank's time."""
    return ws * cell_steps / (ms * 1e-3), ws * cell_steps / t_e2e


def run_ours(args, wl):
    import torch

    from paper_1511_06959_gb300 import api

    ws, rank, local = dist_init()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = api.NS_MIXED if args.precision == "mixed" else api.NS_FP64

    w0_host = wl.initial_state()
    w0 = torch.from_numpy(w0_host).to(dev)
    scheme = api.NS_SSPRK3 if args.scheme == "ssprk3" else api.NS_RK4
    flux = api.NS_FLUX_ROE if args.flux == "roe" else api.NS_FLUX_CENTRAL
    S = api.Solver(wl.nx, wl.ny, wl.nz, wl.dx, gamma=wl.gamma, mu=wl.mu, Pr=wl.Pr, dt=0.0,
                   precision=prec, plane_i=wl.plane_i, pt_in=wl.pt_in, batch=wl.batch, scheme=scheme,
                   flux=flux)
    split = tuple(float(x) for x in args.nu_split.split(","))
    S.set_viscosity_split(*split)
    m = torch.empty(1, dtype=torch.float64, device=dev)
    S.max_wave_speed(w0, m)
    dt = C.cfl_dt(wl, m.item())
    S.set_dt(dt)
    field_bytes = w0.numel() * 8
    param = wl.param if wl.schedule != "revolve" or wl.param else C.revolve_slots(wl, field_bytes)
    sched = C.SCHEDULES[wl.schedule]
    net = None
    if args.closure:
        from paper_1511_06959_gb300 import closure
        net = closure.Network(S, closure.init_params(3, out_bias=0.5))
    run_sched, host, disk = sched, None, None
    if args.disk_snapshots:
        if wl.schedule != "stride":
            raise SystemExit("--disk-snapshots needs a workload with a stride schedule")
        run_sched, disk = api.NS_CKPT_STRIDE_DISK, args.disk_snapshots
    elif args.host_snapshots:
        if wl.schedule != "stride":
            raise SystemExit("--host-snapshots needs a workload with a stride schedule")
        run_sched = api.NS_CKPT_STRIDE_HOST
        probe = S.run_opts(wl.nsteps, run_sched, param)
        host = torch.empty(S.host_bytes(probe), dtype=torch.uint8, pin_memory=True)
    opts = S.run_opts(wl.nsteps, run_sched, param, 0.5 if net is not None else wl.lam_coef, 0.0, True, True,
                      net.blob if net is not None else None, host_arena=host, disk_path=disk)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device=dev)
    J = torch.empty(wl.batch, dtype=torch.float64, device=dev)
    lam0 = torch.empty_like(w0)
    E = torch.empty((wl.nsteps + 1, wl.batch), dtype=torch.float64, device=dev)
    sig = torch.empty((wl.nsteps, wl.batch, 2), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def direct_step():
        S.adjoint_run(w0, opts, arena, J, lam0, energy=E, sigma_stats=sig)

    # The sweep captured once as a CUDA graph (ns_adjoint_run_capture): each step replays
    # all of its kernels from one graph launch, reading w0 as it is then.  The host and disk
    # tiers copy through the host and run the call itself.
    graph = None
    if not args.no_graph and host is None and disk is None:
        graph = S.adjoint_run_capture(w0, opts, arena, J, lam0, energy=E, sigma_stats=sig)
    step = graph.launch if graph is not None else direct_step

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    err = S.last_error()
    if err != 0:
        raise RuntimeError(f"device error word {err} after warm-up")

    bus = torch.cuda.get_device_properties(dev).pci_bus_id if hasattr(
        torch.cuda.get_device_properties(dev), "pci_bus_id") else None
    clk = ClockSampler(bus)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    launches0 = api.launch_count()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)          # L2 flush between timed steps, outside the event pair
        ev[i][0].record()
        step()
        ev[i][1].record()
    torch.cuda.synchronize()
    gl = api.launch_count() - launches0 + (args.steps * graph.kernels if graph is not None else 0)
    if ws > 1:
        torch.distributed.barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # Kernel durations: a second pass of the same K steps with CUDA events recorded by the
    # library on its stream around each step's run of adjoint-stage launches (the event
    # records cost a little, so the headline value comes from the pass without them).
    S.profile_enable(True)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        direct_step()
    torch.cuda.synchronize()
    S.profile_enable(False)
    clocks = clk.stop()
    kms, klaunch = S.profile_read()
    # The same pass with the stride sweep's segments in sequence (ns_set_pipeline off):
    # the adjoint stage alone on the SMs, where in the pipelined sweep it shares them with
    # the concurrent replay of the next segment.
    iso = None
    if wl.schedule == "stride" and host is None and disk is None and wl.nsteps - 1 >= param >= 2:
        S.set_pipeline(False)
        S.profile_enable(True)
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            direct_step()
        torch.cuda.synchronize()
        S.profile_enable(False)
        S.set_pipeline(True)
        iso = S.profile_read()
    if S.last_error() != 0:
        raise RuntimeError("device error word set in the timed region")
    Jv = J.cpu().numpy().copy()
    E_host = E.cpu().numpy()
    if not np.all(np.isfinite(Jv)) or not np.all(np.isfinite(E_host)):
        raise RuntimeError("non-finite objective or adjoint energy")

    # end to end through the public call with host buffers
    w_pin = torch.from_numpy(w0_host).pin_memory()
    lam_pin = torch.empty(lam0.shape, dtype=torch.float64).pin_memory()
    J_pin = torch.empty(wl.batch, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        w0.copy_(w_pin, non_blocking=True)    # the input the sweep (or its graph) reads
        step()
        lam_pin.copy_(lam0, non_blocking=True)
        J_pin.copy_(J, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps

    cell_steps = wl.cells * wl.batch * wl.nsteps
    # max over ranks
    ms, t_e2e = max_over_ranks(ms, t_e2e, ws, dev)
    value, e2e_value = whole_job_rates(ws, cell_steps, ms, t_e2e)

    out = None
    if rank == 0:
        kavg = kms / max(klaunch, 1)
        stages = 3 if args.scheme == "ssprk3" else 4
        ncell = wl.cells * wl.batch
        bytes_launch = ADJ_STEP_BYTES / stages * ncell
        operand_bytes = ADJ_STAGE_OPERAND_BYTES[args.precision] * ncell
        peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
        hbm = peaks.get("hbm_gbs", 6800.0)
        hbm_src = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
        achieved = bytes_launch / (kavg * 1e-3) / 1e9
        sweep_gbs = SWEEP_BYTES * cell_steps / (ms * 1e-3) / 1e9
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 accumulate)" if prec == api.NS_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": C.describe(wl, args.scheme, args.flux), "name": wl.name, "cells": wl.cells,
                       "scheme": args.scheme, "flux": args.flux, "nu_split": list(split),
                       "viscosity": "learned closure (MLP, kappa 0.5)" if args.closure else "sigma_1 rule",
                       "nsteps": wl.nsteps,
                       "schedule": wl.schedule + (" (snapshots in host memory)" if host is not None else
                                                  " (snapshots in a file)" if disk is not None else ""),
                       "param": param,
                       "lambda_tilde": wl.lam_tilde, "precision": args.precision, "dt": dt,
                       "l2": "flushed (256 MB write) between timed steps; arena "
                             f"{arena.numel() / 1e9:.2f} GB > L2",
                       "launch": (f"one CUDA graph launch per sweep ({graph.kernels} kernels, captured once "
                                  "by ns_adjoint_run_capture)" if graph is not None else
                                  "ns_adjoint_run per sweep"),
                       "J_bar": float(Jv[0]), "E_vhat_0": float(E_host[0, 0])},
            "roofline": {"bound": "hbm", "kernel": "k_adj_stage", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": adj_traffic(wl, args.precision),
                         "avg_launch_us": 1e3 * kavg, "launches": klaunch,
                         "kernel_timing": "second K-step pass, CUDA events around each step's adjoint-stage launches"
                                          " (in a pipelined stride sweep the next segment's replay runs on the"
                                          " SMs meanwhile)",
                         "bytes_per_launch": bytes_launch,
                         "bytes_rule": f"{ADJ_STEP_BYTES:.0f} B per adjoint cell-step (read w^n and lam^(n+1), "
                                       f"write lam^n, FP64) / {stages} stage launches",
                         "peak_source": hbm_src,
                         "operand_bytes_per_launch": operand_bytes,
                         "operand_frac": operand_bytes / (kavg * 1e-3) / 1e9 / hbm,
                         "sweep": {"bytes_per_cell_step": SWEEP_BYTES, "achieved": sweep_gbs,
                                   "frac": sweep_gbs / hbm, "unit": "GB/s"},
                         "alu": alu_roofline(wl, args.precision, kavg, api),
                         "isolated": None if iso is None else {
                             "avg_launch_us": 1e3 * iso[0] / max(iso[1], 1),
                             "achieved": bytes_launch / (iso[0] / max(iso[1], 1) * 1e-3) / 1e9,
                             "frac": bytes_launch / (iso[0] / max(iso[1], 1) * 1e-3) / 1e9 / hbm,
                             "alu": alu_roofline(wl, args.precision, iso[0] / max(iso[1], 1), api),
                             "kernel_timing": "the same pass with the segments in sequence "
                                              "(ns_set_pipeline off): no replay shares the SMs"}},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(w0.numel() * 8),
                    "d2h_bytes_per_step": int(lam0.numel() * 8 + J.numel() * 8)},
            "gpu_launches": gl,
            "clocks": clocks,
        }
        if not args.no_fp64_compare and prec == api.NS_MIXED and not args.closure:
            out["fp64"] = fp64_compare(api, torch, wl, w0, dt, sched, param, lam0, Jv, scheme, split, flux)
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(wl, args.scheme, args.flux)
    return out


def alu_roofline(wl, precision, kavg_ms, api):
    """The adjoint-stage kernel against the FP32 (FP64) multiply-add rate measured here:
    achieved = FP32 (FP64) flops per launch, counted by ncu on this kernel source and
    workload (committed summary, hash-checked; None otherwise), over the launch time."""
    kind = api.NS_PEAK_FP64 if precision == "fp64" else None
    try:
        if kind is None:
            peak = max(api.measure_fma_peak(api.NS_PEAK_FP32), api.measure_fma_peak(api.NS_PEAK_FP32X2))
        else:
            peak = api.measure_fma_peak(kind)
    except Exception:
        return None
    flops = adj_profile_field(wl, precision, "fp64_flops_per_launch" if precision == "fp64"
                              else "fp32_flops_per_launch")
    out = {"unit": "TFLOP/s", "peak": peak / 1e12,
           "peak_source": "ns_measure_fma_peak (measured here: best of scalar and paired FMA)"
           if kind is None else "ns_measure_fma_peak (measured here, FP64 FMA)",
           "achieved": None, "frac": None, "flops_per_launch": flops}
    if flops:
        a = flops / (kavg_ms * 1e-3)
        out["achieved"] = a / 1e12
        out["frac"] = a / peak
    return out


ADJ_SOURCES = ("ns_adj.cu", "ns_common.cuh", "ns_kernels.h")
ADJ_PROFILE = os.path.join(ROOT, "profiles", "k_adj_stage_box128_mixed.md")


def adj_source_hash():
    """First 16 hex digits of the SHA-256 of the adjoint stage kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for f in ADJ_SOURCES:
        with open(os.path.join(ROOT, "paper_1511_06959_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def adj_profile_field(wl, precision, key):
    """A per-launch figure of the committed ncu summary of the adjoint-stage kernel, when
    it was taken on this workload and precision from the kernel sources as they are now
    (the summary records their hash); otherwise None."""
    if wl.name != "box128" or precision != "mixed" or not os.path.exists(ADJ_PROFILE):
        return None
    fields = {}
    with open(ADJ_PROFILE) as fh:
        for line in fh:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
    if fields.get("source_sha256_16") != adj_source_hash():
        return None
    try:
        return int(fields[key])
    except (KeyError, ValueError):
        return None


def adj_traffic(wl, precision):
    """DRAM bytes per adjoint-stage launch (ncu, committed summary), or None."""
    return adj_profile_field(wl, precision, "dram_bytes_per_launch")


def fp64_compare(api, torch, wl, w0, dt, sched, param, lam_mixed, J_mixed, scheme, split=(1.0, 1.0, 1.0),
                 flux=0):
    """The same checkpointed sweep in FP64 (timed once) and the mixed-precision
    gradient error against it."""
    S = api.Solver(wl.nx, wl.ny, wl.nz, wl.dx, gamma=wl.gamma, mu=wl.mu, Pr=wl.Pr, dt=dt,
                   precision=api.NS_FP64, plane_i=wl.plane_i, pt_in=wl.pt_in, batch=wl.batch,
                   scheme=scheme, flux=flux)
    S.set_viscosity_split(*split)
    opts = S.run_opts(wl.nsteps, sched, param, wl.lam_coef, 0.0, True, True)
    arena = torch.empty(S.arena_bytes(opts), dtype=torch.uint8, device=w0.device)
    J = torch.empty(wl.batch, dtype=torch.float64, device=w0.device)
    lam = torch.empty_like(w0)
    E = torch.empty((wl.nsteps + 1, wl.batch), dtype=torch.float64, device=w0.device)
    sg = torch.empty((wl.nsteps, wl.batch, 2), dtype=torch.float64, device=w0.device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    S.profile_enable(True)
    a.record()
    S.adjoint_run(w0, opts, arena, J, lam, energy=E, sigma_stats=sg)
    b.record()
    torch.cuda.synchronize()
    S.profile_enable(False)
    ms = a.elapsed_time(b)
    kms, kn = S.profile_read()
    d = (lam_mixed - lam).double()
    rel = (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(lam)).item()
    Jf = J.cpu().numpy()
    return {"value": wl.cells * wl.batch * wl.nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "grad_rel_l2_mixed_vs_fp64": rel,
            "J_rel_mixed_vs_fp64": float(abs(J_mixed[0] - Jf[0]) / abs(Jf[0])),
            "adj_stage_avg_launch_us": 1e3 * kms / max(kn, 1),
            "note": "FP64 is bound by the FP64 ALU rate, not HBM; timed once on the same workload"}


def cpu_baseline(wl, scheme="rk4", flux="central"):
    """The FP64 oracle on this host's cores: one checkpointed adjoint step of the full box
    (forward, replay, stabilised adjoint, source, energy) per process, scaled to adjoint
    cell-steps/s.  First one process alone (single core), then one process per core
    running the same sample at once (all cores: the job's cells over the slowest
    process's time).  The processes are spawned, so no fork happens after CUDA is
    initialised."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    cores = cpu_cores()
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(1) as pool:
            t1 = pool.apply(_cpu_sample, (wl.name, scheme, flux))
        with ctx.Pool(cores) as pool:
            ts = pool.starmap(_cpu_sample, [(wl.name, scheme, flux)] * cores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    tmax = max(ts)
    return {"value": cores * wl.cells * wl.batch / tmax, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes at once, each 1 checkpointed adjoint step (forward + replay + "
                      f"stabilised adjoint + source + energy) of the full {wl.nx}x{wl.ny}x{wl.nz} box, numpy "
                      f"FP64, one BLAS thread each; slowest {tmax:.1f} s",
            "single_core": {"value": wl.cells * wl.batch / t1, "cores": 1, "seconds": t1},
            "host_cores_available": cores}


def _cpu_sample(name, scheme="rk4", flux="central"):
    wl = C.WORKLOADS[name]
    w, P = oracle_setup(wl, scheme, flux)
    t0 = time.perf_counter()
    oracle_unit(w, P, wl.lam_tilde, wl.dx[0])
    return time.perf_counter() - t0


def main():
    args = parse()
    wl = C.WORKLOADS[args.workload]
    if args.nsteps > 0:
        import dataclasses
        wl = dataclasses.replace(wl, nsteps=args.nsteps)
    if args.impl == "reference":
        run_reference(args, wl)
        return
    out = run_ours(args, wl)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

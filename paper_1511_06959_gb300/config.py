"""Named workloads and their derived solver parameters.

Units: free stream rho = 1, p = 1/gamma (sound speed 1), velocity = Mach number, box
length along x = 1; mu = rho U L / Re with U the mean speed and L the x length.
The pressure-loss plane is the x-face at 0.75 L_x; p_t,in is the stagnation pressure of
the mean flow (the periodic box has no inlet).
"""
from __future__ import annotations

import dataclasses

from . import synth


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    kind: str            # "vortex" or "turbulence"
    mach: float
    Re: float
    nsteps: int
    schedule: str        # "all", "stride", "revolve"
    param: int = 0       # stride, or revolve slots (0: from budget_gb)
    budget_gb: float = 0.0
    rms: float = 0.0
    seed: int = 1
    batch: int = 1
    lam_tilde: float = 0.0   # adjoint viscosity nu = lam_tilde dx^2 sigma_1
    gamma: float = 1.4
    Pr: float = 0.72
    cfl: float = 0.5

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dx(self):
        return synth.box_shape(self.nx, self.ny, self.nz)

    @property
    def mu(self) -> float:
        return self.mach * 1.0 / self.Re

    @property
    def plane_i(self) -> int:
        return (3 * self.nx) // 4

    @property
    def pt_in(self) -> float:
        g = self.gamma
        return (1.0 / g) * (1.0 + 0.5 * (g - 1.0) * self.mach ** 2) ** (g / (g - 1.0))

    @property
    def lam_coef(self) -> float:
        return self.lam_tilde * self.dx[0] ** 2

    def initial_state(self):
        if self.kind == "vortex":
            return synth.isentropic_vortex(self.nx, self.ny, self.nz, mach=self.mach, noise=1e-3,
                                           seed=self.seed, gamma=self.gamma)
        return synth.solenoidal_turbulence(self.nx, self.ny, self.nz, mach=self.mach, rms=self.rms,
                                           seed=self.seed, gamma=self.gamma)


WORKLOADS = {
    # 2D vortex box, all states kept
    "vortex64": Workload("vortex64", 64, 64, 1, "vortex", 0.5, 1e3, 200, "all", seed=1),
    # 3D transonic turbulent box, a snapshot every 50 steps
    "box128": Workload("box128", 128, 64, 64, "turbulence", 0.9, 1e4, 1000, "stride", param=50,
                       rms=0.10, seed=2, lam_tilde=0.1),
    # z-aligned vortex columns, the autograd and closure-judging size (8 boxes in a batch)
    "column96": Workload("column96", 96, 48, 48, "vortex", 0.5, 1e3, 100, "all", seed=3, batch=8),
    # large transonic box, binomial checkpointing inside a 60 GB budget (500-step window)
    "box512": Workload("box512", 512, 256, 128, "turbulence", 0.9, 5e4, 500, "revolve",
                       budget_gb=60.0, rms=0.08, seed=4, lam_tilde=0.1),
}


def revolve_slots(w: Workload, field_bytes: int) -> int:
    """State slots that fit the workload's HBM budget next to the sweep's fixed fields."""
    fixed = 3 * field_bytes + 2 * w.cells * w.batch * 4
    return max(1, int((w.budget_gb * 1e9 - fixed) // field_bytes))


def cfl_dt(w: Workload, max_wave_speed: float) -> float:
    return w.cfl * min(w.dx) / max_wave_speed


def describe(w: Workload, scheme: str = "rk4", flux: str = "central") -> str:
    name = "SSP-RK3" if scheme == "ssprk3" else "RK4"
    fl = ", Roe flux" if flux == "roe" else ""
    return (f"{w.nx}x{w.ny}x{w.nz} {w.kind} Mach {w.mach} Re {w.Re:g}, {w.nsteps} {name} steps{fl}, "
            f"{w.schedule}{'' if w.schedule == 'all' else ' ' + str(w.param or 'budget')}")


SCHEDULES = {"all": 0, "stride": 1, "revolve": 2}

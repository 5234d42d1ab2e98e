"""Seeded synthetic inputs: electron super-particles of a uniform Maxwellian shell.

This module holds no arithmetic of the method itself (no field, no push): it
draws the initial state that the CUDA path and the CPU oracle both start from.

Recipe (dimensionless units of Sec. 4: lengths in R, velocities in R*omega_pe):
  * positions uniform in the shell 1 <= r <= r_out: r = (1 + u (r_out^3 - 1))^(1/3)
    with an isotropic direction (normalised Gaussian 3-vector);
  * velocities: each Cartesian component normal with standard deviation
    lambda_D / R (thermal speed lambda_D omega_pe);
  * every value is rounded to float32 and stored as float64, so the FP64 and the
    mixed-precision paths start from bit-identical states;
  * the radius is kept a relative 1e-6 inside both walls after rounding.
The generator is numpy's Philox bit generator keyed by the seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12
M_E = 9.1093837015e-31


def debye_length_m(n_e_m3: float, T_e_eV: float) -> float:
    return float(np.sqrt(EPS0 * T_e_eV / (n_e_m3 * E_CHARGE)))


@dataclass
class Workload:
    """A physical configuration of the probe, the plasma and the run."""
    name: str
    N: int
    l_max: int
    T_e_eV: float
    n_e_m3: float
    R_E_m: float = 4e-3
    R_D_m: float = 5e-3
    eps_D: float = 4.0
    outer_debye: float = 20.0          # outer wall at R_D + outer_debye * lambda_D
    outer_R: float = 0.0               # if > 0: outer wall at outer_R * R_D instead
    dt: float = 0.05
    steps: int = 2000
    drive_kind: int = 0                # 0 Gaussian pulse, 1 impulse, 2 off
    V_volts: float = 1.0
    width_wpe: float = 2.0
    precision: int = 0                 # 0 FP64, 1 mixed
    seed: int = 0
    wall_rule: int = 0
    self_image: int = 0
    m0_only: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def R_out_m(self) -> float:
        if self.outer_R > 0:
            return self.outer_R * self.R_D_m
        return self.R_D_m + self.outer_debye * debye_length_m(self.n_e_m3, self.T_e_eV)

    @property
    def r_out(self) -> float:
        return self.R_out_m / self.R_D_m

    @property
    def sigma_v(self) -> float:
        return debye_length_m(self.n_e_m3, self.T_e_eV) / self.R_D_m


# The single-instance workloads: a small FP64 case, the mixed-precision case at
# N = 2e6 / l_max = 16, and the large roofline case at N = 1.6e7 / l_max = 24.
WORKLOADS = {
    "fp64_n2e4_l8": Workload("fp64_n2e4_l8", N=20000, l_max=8, T_e_eV=2.0, n_e_m3=1e15,
                             steps=2000, precision=0, seed=0),
    "mixed_n2e6_l16": Workload("mixed_n2e6_l16", N=2000000, l_max=16, T_e_eV=3.0, n_e_m3=1e16,
                               steps=20000, precision=1, seed=0),
    # profiling size of the l_max = 24 case (a few GB on the device)
    "mixed_n4e6_l24": Workload("mixed_n4e6_l24", N=4000000, l_max=24, T_e_eV=2.0, n_e_m3=1e16,
                               outer_debye=40.0, steps=5000, precision=1, seed=0),
    "mixed_n1.6e7_l24": Workload("mixed_n1.6e7_l24", N=16000000, l_max=24, T_e_eV=2.0,
                                 n_e_m3=1e16, outer_debye=40.0, steps=5000, precision=1, seed=0),
}


def paper_variant(T_e_eV: float, N: int = 500000, steps: int = 10000, seed: int = 0) -> Workload:
    """The paper's own case (Sec. 4): probe radius R = 4 mm with a 1 mm dielectric
    (R_E = 3 mm), n = 1e15 m^-3, domain 1 < r < 10, the l <= 1, m = 0 kernel
    (Sec. 3), a single kick u_asy = 1 at the first step (289 V in the units
    eps0 V / (n e R^2) = u), dt = 0.01. The plasma here is the uniform
    Maxwellian shell, not the paper's sheath equilibrium (App. D), and
    eps_D = 4 (the paper does not state it)."""
    return Workload(f"paper_m0_l1_T{T_e_eV:g}", N=N, l_max=1, T_e_eV=T_e_eV, n_e_m3=1e15,
                    R_E_m=3e-3, R_D_m=4e-3, eps_D=4.0, outer_R=10.0, dt=0.01, steps=steps,
                    drive_kind=1, V_volts=289.0, precision=1, seed=seed, m0_only=1)


def maxwellian_shell(N: int, r_out: float, sigma_v: float, seed: int = 0,
                     r_in: float = 1.0):
    """Returns (x [N,3], v [N,3]) float64 arrays holding float32 values."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    u = rng.random(N)
    lo = r_in * (1.0 + 1e-6)
    hi = r_out * (1.0 - 1e-6)
    r = np.cbrt(lo ** 3 + u * (hi ** 3 - lo ** 3))
    d = rng.standard_normal((N, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    x = (d * r[:, None]).astype(np.float32).astype(np.float64)
    # re-project rounded points that drifted outside the shell
    rr = np.linalg.norm(x, axis=1)
    bad = (rr < lo) | (rr > hi)
    if np.any(bad):
        x[bad] = (x[bad] / rr[bad, None] * np.clip(rr[bad], lo, hi)[:, None]).astype(np.float32)
    v = (rng.standard_normal((N, 3)) * sigma_v).astype(np.float32).astype(np.float64)
    return np.ascontiguousarray(x), np.ascontiguousarray(v)


def radial_profile_shell(N: int, r_grid, cum, sigma_v: float, seed: int = 0):
    """Returns (x [N,3], v [N,3]) like maxwellian_shell, with radii drawn from a
    given radial distribution instead of the uniform one: cum[k] is the
    (unnormalised, non-decreasing) number of particles inside r_grid[k], taken
    linear between nodes, so a radius is the inverse of that piecewise-linear
    function at a uniform fraction of cum[-1]. The table is an input (e.g. the
    electron charge of an equilibrium profile); nothing here computes it."""
    r_grid = np.asarray(r_grid, dtype=np.float64)
    cum = np.asarray(cum, dtype=np.float64)
    rng = np.random.Generator(np.random.Philox(key=seed))
    u = rng.random(N)
    lo = r_grid[0] * (1.0 + 1e-6)
    hi = r_grid[-1] * (1.0 - 1e-6)
    r = np.clip(np.interp(u * cum[-1], cum, r_grid), lo, hi)
    d = rng.standard_normal((N, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    x = (d * r[:, None]).astype(np.float32).astype(np.float64)
    rr = np.linalg.norm(x, axis=1)
    bad = (rr < lo) | (rr > hi)
    if np.any(bad):
        x[bad] = (x[bad] / rr[bad, None] * np.clip(rr[bad], lo, hi)[:, None]).astype(np.float32)
    v = (rng.standard_normal((N, 3)) * sigma_v).astype(np.float32).astype(np.float64)
    return np.ascontiguousarray(x), np.ascontiguousarray(v)


def workload_state(w: Workload, N: int | None = None):
    """Initial state of a workload (optionally with a different particle count)."""
    return maxwellian_shell(w.N if N is None else N, w.r_out, w.sigma_v, w.seed)

"""Floating probe-plasma equilibrium of App. D (the initial condition of the
simulation), written out with scipy. Test infrastructure: only tests, the
smoke check and the CPU baseline of the benchmark use it.

Units as in Sec. 4: r in R (probe radius), densities in n_inf, psi = e Phi / T_e,
lambda = lambda_D / R. The appendix's equations then read

  Poisson (App. D):   lambda^2 (1/r^2) d/dr (r^2 dpsi/dr) = n_e - n_i
  Boltzmann electrons: n_e = exp(psi)
  ions from infinity:  n_i = Rhat^2 / (r^2 sqrt(-2 psi))
  (constant radial ion flux 4 pi Rhat^2 n_inf c_s, energy conservation
   m_i v^2 / 2 + e Phi = 0, c_s = sqrt(T_e/m_i))
  floating condition (Hertz-Langmuir electron flux = ion flux at r = 1):
     Rhat^2 = sqrt(m_i / (2 pi m_e)) exp(psi(1)).

Far from the probe the plasma is quasi-neutral: exp(psi) = n_i, i.e.
psi + ln(-2 psi)/2 = 2 ln(Rhat / r), the branch with -1/2 < psi < 0 (it
ends at the Bohm point psi = -1/2, r_B = Rhat e^{1/4}).

Shooting (App. D): for a trial Rhat, start on the quasi-neutral branch at the
outer radius r_out of the domain (value and slope of the branch there) and
integrate Poisson's equation inwards to r = 1; Rhat is the root of the
floating condition psi(1; Rhat) = 2 ln Rhat - ln sqrt(m_i/(2 pi m_e)).
Reading: the appendix puts psi = 0 at infinity and names no starting radius;
starting at r_out neglects the Poisson correction of the quasi-neutral branch
beyond the domain, which is of order lambda^2 / r^2 there.

Alongside psi the integration carries the charges outside r (in n_inf R^3):
A_i(r) = int_r^{r_out} 4 pi s^2 n_i ds and A_e likewise, so that the charge
inside r is A(1) - A(r). Gauss's law at the probe gives the surface charge
Q_S = -4 pi lambda^2 psi'(1) (units n_inf R^3 e; negative for a floating probe).
"""
import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq


def floating_constant(mass_ratio):
    """ln sqrt(m_i / (2 pi m_e)) of the floating condition (App. D)."""
    return 0.5 * np.log(mass_ratio / (2.0 * np.pi))


def psi_qn(r, rhat):
    """Quasi-neutral potential exp(psi) = Rhat^2 / (r^2 sqrt(-2 psi)) on its
    branch -1/2 < psi < 0 (exists for r > Rhat e^{1/4}); by bracketing."""
    t = 2.0 * np.log(rhat / r)
    if t >= -0.5:
        raise ValueError("r inside the Bohm radius: no quasi-neutral solution")

    def g(p):
        return p + 0.5 * np.log(-2.0 * p) - t

    # g falls on (-1/2, 0) from -1/2 - t > 0 to -inf; at p = -e^{2t}/2 it is
    # -e^{2t}/2 < 0, so the root lies between -1/2 and that point
    hi = -min(0.25, 0.5 * np.exp(2.0 * t))
    while g(hi) > 0:
        hi *= 1e-3
    return brentq(g, -0.5, hi, xtol=1e-300, rtol=1e-15, maxiter=1000)


def dpsi_qn(r, rhat):
    """Radial slope of the quasi-neutral branch: differentiating
    psi + ln(-2 psi)/2 = 2 ln(Rhat/r) gives psi' (1 + 1/(2 psi)) = -2/r."""
    p = psi_qn(r, rhat)
    return -2.0 / (r * (1.0 + 1.0 / (2.0 * p)))


def shoot(rhat, lam, r_out, dense=False, rtol=1e-11):
    """Integrates Poisson's equation inwards from the quasi-neutral branch at
    r_out to r = 1. State: psi, psi', A_i, A_e. Returns the solve_ivp result."""
    p0 = psi_qn(r_out, rhat)
    d0 = dpsi_qn(r_out, rhat)
    lam2 = lam * lam

    def rhs(r, y):
        psi, dp = y[0], y[1]
        ni = rhat * rhat / (r * r * np.sqrt(-2.0 * psi))
        ne = np.exp(psi)
        return [dp, (ne - ni) / lam2 - 2.0 * dp / r, -4.0 * np.pi * r * r * ni,
                -4.0 * np.pi * r * r * ne]

    return solve_ivp(rhs, (r_out, 1.0), [p0, d0, 0.0, 0.0], method="DOP853", rtol=rtol,
                     atol=[1e-16, 1e-13, 1e-12, 1e-12], dense_output=dense)


def floating_residual(rhat, lam, mass_ratio, r_out):
    """psi(1; Rhat) - (2 ln Rhat - ln sqrt(m_i/(2 pi m_e))): positive for too
    small Rhat (no sheath yet), negative for too large."""
    s = shoot(rhat, lam, r_out)
    return s.y[0, -1] - 2.0 * np.log(rhat) + floating_constant(mass_ratio)


def equilibrium(lam, mass_ratio, r_out, n_grid=1025):
    """The floating equilibrium on the uniform grid r_k = 1 + k (r_out-1)/(n_grid-1).

    Returns a dict: rhat, psi_wall = psi(1), dpsi_wall = psi'(1), q_s (App. D
    surface charge, n_inf R^3 e), r, psi, q_ion and q_elec (charge inside r_k),
    n_ion = Rhat^2/(r^2 sqrt(-2 psi)), n_elec = exp(psi)."""
    lo = 0.5 * np.exp(-0.25)
    hi = 2.0
    while floating_residual(hi, lam, mass_ratio, r_out) > 0:
        hi *= 1.5
        if hi * np.exp(0.25) >= r_out:
            raise ValueError("no floating equilibrium inside r_out")
    rhat = brentq(floating_residual, lo, hi, args=(lam, mass_ratio, r_out), xtol=1e-15,
                  rtol=1e-14, maxiter=200)
    s = shoot(rhat, lam, r_out, dense=True)
    r = 1.0 + (r_out - 1.0) * np.arange(n_grid) / (n_grid - 1)
    r[-1] = r_out
    y = s.sol(r)
    y[:, -1] = [psi_qn(r_out, rhat), dpsi_qn(r_out, rhat), 0.0, 0.0]
    y[:, 0] = s.y[:, -1]
    psi = y[0]
    q_ion = y[2, 0] - y[2]
    q_elec = y[3, 0] - y[3]
    return dict(rhat=rhat, psi_wall=s.y[0, -1], dpsi_wall=s.y[1, -1],
                q_s=-4.0 * np.pi * lam * lam * s.y[1, -1], r=r, psi=psi, dpsi=y[1],
                q_ion=q_ion, q_elec=q_elec,
                n_ion=rhat * rhat / (r * r * np.sqrt(-2.0 * psi)), n_elec=np.exp(psi))

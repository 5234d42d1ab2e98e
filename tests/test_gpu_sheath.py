"""The simulation started from the floating equilibrium of App. D: immobile
ions of the equilibrium's radial profile, its surface charge, electrons drawn
from its Boltzmann density. Field and steps against the oracle with the same
ion table, and the equilibrium kept by the electrons' own dynamics."""
import numpy as np
import pytest

import oracle
from paper_2111_13072_gb300.inputs import Workload, radial_profile_shell

pytestmark = pytest.mark.gpu

from parity_metrics import TOL, check_field
ARGON = 39.948 * 1822.888486
# the paper's probe and plasma (Sec. 4): R = 4 mm, R_E = 3 mm, n = 1e15 m^-3, T_e = 3 eV, r < 10 R
PAPER = Workload("sheath", N=3000, l_max=8, T_e_eV=3.0, n_e_m3=1e15, R_E_m=3e-3, R_D_m=4e-3,
                 eps_D=4.0, outer_R=10.0, dt=0.01, drive_kind=2)


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available(), "these tests need the GPU"
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


@pytest.fixture(scope="module")
def eq(imrp):
    lam = oracle.debye_length(PAPER.n_e_m3, PAPER.T_e_eV) / PAPER.R_D_m
    return lam, imrp.sheath_solve(lam, ARGON, PAPER.outer_R, 2049)


def _pair(imrp, eq, n, **over):
    lam, e = eq
    p = imrp.params_from_workload(PAPER, N=n, **over)
    op = oracle.from_physical(PAPER.R_E_m, PAPER.R_D_m, PAPER.eps_D, PAPER.R_out_m, PAPER.n_e_m3,
                              PAPER.T_e_eV, n, p.l_max, p.dt, drive_kind=p.drive_kind,
                              V_volts=p.V_volts, width_wpe=p.width_wpe, wall_rule=p.wall_rule,
                              self_image=p.self_image, seed=p.seed)
    # the same ions and surface charge in super-particle charges: n~ = N / Q_e
    op.n_tilde = n / e["q_elec"][-1]
    op.ion_q = e["q_ion"] * op.n_tilde
    op.q_s = e["q_s"] * op.n_tilde
    op.n_ion = 0.0
    return p, op


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,L,drive", [(3000, 8, 2), (1057, 4, 1)])
def test_field_with_ion_profile_matches_oracle(imrp, eq, prec, n, L, drive):
    lam, e = eq
    x, v = radial_profile_shell(n, e["r"], e["q_elec"], lam, seed=11)
    p, op = _pair(imrp, eq, n, precision=prec, l_max=L, drive_kind=drive, V_volts=289.0)
    with imrp.Sim(p) as sim:
        sim.set_ion_profile(e["q_ion"], e["q_elec"][-1], e["q_s"])
        sim.load(x, v)
        E = sim.field()
    Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
    check_field(E, Eo, prec, f"ion profile n={n} L={L}")


@pytest.mark.parametrize("prec", [0, 1])
def test_steps_with_ion_profile_match_oracle(imrp, eq, prec):
    lam, e = eq
    n = 2000
    x, v = radial_profile_shell(n, e["r"], e["q_elec"], lam, seed=12)
    p, op = _pair(imrp, eq, n, precision=prec, l_max=4, dt=0.05)
    with imrp.Sim(p) as sim:
        sim.load(x, v)                      # the profile may also come after the load
        sim.set_ion_profile(e["q_ion"], e["q_elec"][-1], e["q_s"])
        q, u = sim.step(4)
        xg, vg = sim.particles()
    xo, vo, qo, uo, hits = oracle.run(op, x, v, 4)
    dv_g, dv_o = vg - v, vo - v
    per = np.linalg.norm(dv_g - dv_o, axis=1) / (np.linalg.norm(dv_o, axis=1) + 1e-30)
    good = per <= 10 * TOL[prec]
    # a wall hit draws its new direction from the same counter; rounding can move one particle
    assert np.sum(~good) <= (0 if prec == 0 else 2)
    assert _rel(dv_g[good], dv_o[good]) < 10 * TOL[prec]
    assert _rel(xg[good], xo[good]) < TOL[prec]


def test_profile_can_be_switched_off(imrp, eq):
    """n_tab = 0 restores the uniform background and the parameters' Q_S."""
    lam, e = eq
    n = 1500
    x, v = radial_profile_shell(n, e["r"], e["q_elec"], lam, seed=13)
    p = imrp.params_from_workload(PAPER, N=n)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        E0 = sim.field()
        sim.set_ion_profile(e["q_ion"], e["q_elec"][-1], e["q_s"])
        E1 = sim.field()
        sim.set_ion_profile(None, 1.0, 0.0)
        E2 = sim.field()
        with pytest.raises(imrp.IMRPError):
            sim.set_ion_profile(e["q_ion"][::-1], e["q_elec"][-1], e["q_s"])  # decreasing
    np.testing.assert_allclose(E2, E0, rtol=1e-12, atol=0)
    # ions and surface charge of the sheath against the uniform background (at N = 1500 the
    # pair field is noisy, so the l = 0 change is a few per cent of the whole)
    assert _rel(E1, E0) > 0.02


def _radial_counts(x, edges):
    return np.histogram(np.linalg.norm(x, axis=1), edges)[0].astype(np.float64)


def test_equilibrium_is_kept(imrp, eq):
    """Started from the equilibrium, the electrons' radial profile stays put over
    several plasma periods (counts within 5 standard deviations); with the
    uniform background instead the electrons flood the sheath."""
    lam, e = eq
    n = 1000000
    x, v = radial_profile_shell(n, e["r"], e["q_elec"], lam, seed=14)
    edges = np.array([1.0, 1.3, 1.5, 1.8, 2.2, 3.0, 4.5, 7.0, 10.0])
    c0 = _radial_counts(x, edges)
    out = {}
    for profile in (True, False):
        p = imrp.params_from_workload(PAPER, N=n, precision=1, l_max=4, dt=0.05)
        with imrp.Sim(p) as sim:
            if profile:
                sim.set_ion_profile(e["q_ion"], e["q_elec"][-1], e["q_s"])
            sim.load(x, v)
            sim.step(400)                  # t = 20 / omega_pe, about three plasma periods
            xg, _ = sim.particles()
        out[profile] = _radial_counts(xg, edges)
    assert np.all(np.abs(out[True] - c0) < 5 * np.sqrt(c0) + 3), (c0, out[True])
    assert out[False][0] > 2 * c0[0] + 5 * np.sqrt(c0[0]), (c0, out[False])

"""Pins of the oracle's floating equilibrium (App. D) and of its immobile-ion
profile in the field, against limits and laws that the solver does not use
directly. CPU only."""
import numpy as np
import pytest

import oracle
from oracle import sheath as S

ARGON = 39.948 * 1822.888486  # m_i / m_e for argon


@pytest.fixture(scope="module")
def eq_paper():
    # the paper's Fig. 5 setting: n_inf = 1e15 m^-3, T_e = 3 eV, R = 4 mm -> lambda_D / R = 0.1018
    lam = oracle.debye_length(1e15, 3.0) / 4e-3
    return lam, S.equilibrium(lam, ARGON, 10.0, n_grid=2049)


def test_quasi_neutral_branch_solves_its_equation():
    # pick psi on (-1/2, 0) and put r where exp(psi) sqrt(-2 psi) = Rhat^2 / r^2
    rhat = 1.3
    for psi in (-0.49, -0.3, -0.05, -1e-3, -1e-7):
        r = rhat * np.exp(-psi / 2) * (-2 * psi) ** -0.25
        assert S.psi_qn(r, rhat) == pytest.approx(psi, rel=1e-12)
    # slope against a centred difference of the branch
    r, h = 3.0, 1e-5
    fd = (S.psi_qn(r + h, rhat) - S.psi_qn(r - h, rhat)) / (2 * h)
    assert S.dpsi_qn(r, rhat) == pytest.approx(fd, rel=1e-7)


def test_thin_sheath_limit_is_the_planar_floating_probe():
    # lambda -> 0: the sheath shrinks onto the probe, the Bohm point r_B = Rhat e^{1/4}
    # tends to 1, so Rhat -> e^{-1/4} and psi(1) -> -1/2 - ln sqrt(m_i/(2 pi m_e)),
    # the textbook floating potential of a planar probe (-5.18 for argon)
    dev, gap = [], []
    psi_f = -0.5 - S.floating_constant(ARGON)
    assert psi_f == pytest.approx(-5.1789, abs=1e-3)
    for lam in (0.01, 0.005):
        e = S.equilibrium(lam, ARGON, 3.0, n_grid=65)
        dev.append(e["rhat"] / np.exp(-0.25) - 1.0)
        gap.append(e["psi_wall"] - psi_f)
    assert 0 < dev[1] < dev[0] < 0.15
    # the sheath thickness scales as a power of lambda between 1/2 and 1
    assert 2 ** 0.5 < dev[0] / dev[1] < 2.0
    assert 0 < gap[1] < gap[0] < 0.25


def test_gauss_law_and_floating_condition(eq_paper):
    lam, e = eq_paper
    r = e["r"]
    # charge inside r (surface charge + ions - electrons) against the field there
    q_in = e["q_s"] + e["q_ion"] - e["q_elec"]
    e_field = -4 * np.pi * lam ** 2 * r ** 2 * e["dpsi"]
    assert np.max(np.abs(q_in - e_field)) < 1e-8 * np.max(np.abs(e["q_ion"]))
    # Hertz-Langmuir flux balance
    assert e["rhat"] ** 2 == pytest.approx(np.sqrt(ARGON / (2 * np.pi)) * np.exp(e["psi_wall"]),
                                           rel=1e-10)
    # the probe floats negative: negative surface charge, psi rising outwards
    assert e["q_s"] < 0 and e["psi_wall"] < -3.0
    assert np.all(np.diff(e["psi"]) > 0)
    # a positive space-charge sheath at the probe, quasi-neutral plasma far out
    assert e["n_ion"][1] > 2 * e["n_elec"][1]


def test_far_plasma_follows_the_quasi_neutral_branch(eq_paper):
    lam, e = eq_paper
    for rr in (5.0, 7.0, 9.0):
        k = int(np.argmin(np.abs(e["r"] - rr)))
        qn = S.psi_qn(e["r"][k], e["rhat"])
        # the Poisson correction is of order lambda^2 / r^2 relative
        assert abs(e["psi"][k] - qn) < 10 * lam ** 2 / e["r"][k] ** 2 * abs(qn)
    # the densities match there too
    k = int(np.argmin(np.abs(e["r"] - 6.0)))
    assert e["n_ion"][k] == pytest.approx(e["n_elec"][k], rel=1e-3)


def test_charge_tables_integrate_the_densities(eq_paper):
    lam, e = eq_paper
    r = e["r"]
    # trapezoid of 4 pi r^2 n over the fine grid against the carried integrals
    for n, q in ((e["n_ion"], e["q_ion"]), (e["n_elec"], e["q_elec"])):
        f = 4 * np.pi * r ** 2 * n
        trap = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(r))])
        assert np.max(np.abs(trap - q)) < 2e-4 * q[-1]


def test_ion_profile_field_matches_the_uniform_background():
    # a fine table of the uniform background's charge reproduces its field and
    # potential up to the linear interpolation error
    rng = np.random.default_rng(3)
    n = 64
    r_out = 4.0
    rr = rng.uniform(1.0, r_out, n) ** 1.0
    u = rng.normal(size=(n, 3))
    x = (u / np.linalg.norm(u, axis=1, keepdims=True)) * rr[:, None]
    v = rng.normal(size=(n, 3)) * 0.1
    vsh = 4 * np.pi / 3 * (r_out ** 3 - 1)
    p = oracle.Params(d=0.2, eps=4.0, r_out=r_out, n_tilde=n / vsh, n_ion=float(n), L=4)
    grid = np.linspace(1.0, r_out, 4001)
    pt = oracle.Params(d=0.2, eps=4.0, r_out=r_out, n_tilde=n / vsh, n_ion=0.0, L=4,
                       ion_q=n * (grid ** 3 - 1) / (r_out ** 3 - 1))
    e0 = oracle.field_brute(p, x)
    e1 = oracle.field_brute(pt, x)
    scale = np.max(np.abs(e0))
    assert np.max(np.abs(e1 - e0)) < 1e-6 * scale
    assert oracle.energy(pt, x, v) == pytest.approx(oracle.energy(p, x, v), rel=1e-6)

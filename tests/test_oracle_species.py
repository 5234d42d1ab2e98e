"""Pins of the oracle with mobile ions as particles (the paper moves its ions,
Sec. 4): per-particle charge and mass. Against brute force, the Hamiltonian
of Sec. 2 (its gradient and its conservation), charge conjugation, and the
electron-only results. CPU only."""
import numpy as np
import pytest

import oracle
from paper_2111_13072_gb300.inputs import maxwellian_shell


def _mixed(n=48, L=4, seed=5, frac_ion=0.4, m_ion=50.0):
    x, v = maxwellian_shell(n, 2.6, 0.02, seed=seed, r_in=1.4)
    rng = np.random.default_rng(seed)
    ion = rng.random(n) < frac_ion
    q = np.where(ion, 1.0, -1.0)
    m = np.where(ion, m_ion, 1.0)
    v[ion] /= np.sqrt(m_ion)  # thermal ions
    p = oracle.Params(d=0.2, eps=4.0, r_out=3.5, n_tilde=10.0, n_ion=0.0, L=L, wall_rule=1,
                      drive_kind=2, charge=q, mass=m)
    return p, x, v, ion


@pytest.mark.parametrize("si,m0,L", [(0, 0, 6), (1, 0, 4), (0, 1, 3)])
def test_scan_matches_brute_force_with_ions(si, m0, L):
    p, x, v, ion = _mixed(n=300, L=L, seed=2)
    p.self_image, p.m0_only, p.q_s = si, m0, 0.8
    Eb = oracle.field_brute(p, x, u=0.2)
    Es = oracle.field_scan(p, x, u=0.2)
    assert np.linalg.norm(Es - Eb) < 1e-10 * np.linalg.norm(Eb)


def test_explicit_electrons_reproduce_the_default():
    p, x, v, _ = _mixed(n=200, L=4, seed=3)
    n = len(x)
    pe = oracle.Params(d=p.d, eps=p.eps, r_out=p.r_out, n_tilde=p.n_tilde, n_ion=float(n), L=4,
                       wall_rule=0, drive_kind=0, v_hat=0.05, seed=4, nu_coll=0.3)
    pq = oracle.Params(d=p.d, eps=p.eps, r_out=p.r_out, n_tilde=p.n_tilde, n_ion=float(n), L=4,
                       wall_rule=0, drive_kind=0, v_hat=0.05, seed=4, nu_coll=0.3,
                       charge=-np.ones(n), mass=np.ones(n))
    np.testing.assert_array_equal(oracle.field_scan(pq, x, u=0.1), oracle.field_scan(pe, x, u=0.1))
    assert oracle.energy(pq, x, v, u=0.1) == oracle.energy(pe, x, v, u=0.1)
    a = oracle.run(pe, x.copy(), v.copy(), 5)
    b = oracle.run(pq, x.copy(), v.copy(), 5)
    for ya, yb in zip(a, b):
        np.testing.assert_array_equal(np.asarray(ya), np.asarray(yb))


def test_charge_conjugation_reverses_the_particle_field():
    """Without external charges (no ion background, no Q_S, no drive) the field
    is linear in the charges: all charges flipped, the field flips exactly."""
    p, x, v, _ = _mixed(n=120, L=5, seed=6)
    E = oracle.field_scan(p, x)
    p.charge = -p.charge
    np.testing.assert_array_equal(oracle.field_scan(p, x), -E)
    # Q_diff is linear in the charges as well
    q1 = oracle.qdiff(p, x)
    p.charge = -p.charge
    assert oracle.qdiff(p, x) == pytest.approx(-q1, rel=1e-14)


@pytest.mark.parametrize("si,qs,u", [(0, 0.0, 0.0), (1, 0.7, 0.3)])
def test_force_is_energy_gradient_with_ions(si, qs, u):
    """q_k E_k = -grad_k H for electrons and ions alike (Sec. 2 Hamiltonian
    with the charges in the pair, self-image, background and drive terms)."""
    p, x, v, ion = _mixed()
    p.self_image, p.q_s = si, qs
    E = oracle.field_brute(p, x, u=u)
    h = 1e-6
    ks = [int(np.flatnonzero(ion)[0]), int(np.flatnonzero(ion)[1]), int(np.flatnonzero(~ion)[0]), 47]
    for k in ks:
        g = np.zeros(3)
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            g[c] = (oracle.energy(p, xp, v, u=u) - oracle.energy(p, xm, v, u=u)) / (2 * h)
        np.testing.assert_allclose(p.charge[k] * E[k], -g, rtol=1e-6, atol=1e-9)


def test_energy_conservation_with_ions():
    """Drive off, specular walls, ions 50 times heavier: H (kinetic sum
    m v^2 / 2) is conserved to a small fraction of the energy exchanged, and
    the error falls with dt. (Opposite charges cross radii often; the kink of
    the 1/r_> kernel there makes the error first order in dt.)"""

    def worst_error(dt, T=4.0):
        p, x, v, ion = _mixed(n=48, L=4, seed=8)
        p.dt = dt
        qm = (p.charge / p.mass)[:, None]
        H0 = oracle.energy(p, x, v)
        K0 = 0.5 * np.sum(p.mass[:, None] * v * v)
        chunk = int(round(T / dt)) // 8
        worst, dK, first = 0.0, 0.0, True
        for c in range(8):
            x, v, _, _, hits = oracle.run(p, x, v, chunk, step0=c * chunk, first_half_kick=first)
            first = False
            assert hits == 0
            E = oracle.field_scan(p, x)
            vs = v - 0.5 * dt * qm * E  # velocities synchronous with x
            worst = max(worst, abs(oracle.energy(p, x, vs) - H0))
            dK = max(dK, abs(0.5 * np.sum(p.mass[:, None] * vs * vs) - K0))
        return worst, dK

    w1, dK1 = worst_error(0.025)
    w2, dK2 = worst_error(0.0125)
    assert dK2 > 0.5 * dK1 > 0
    assert w2 < 0.01 * dK2
    assert w2 < 0.7 * w1


def test_first_kick_uses_charge_over_mass():
    """From velocities synchronous with x the first kick is dt/2 (q/m) E(x0):
    ions are pushed the other way and m_i times less."""
    p, x, v, ion = _mixed(n=60, L=4, seed=9)
    p.dt = 0.01
    E = oracle.field_scan(p, x)
    x1, v1, _, _, hits = oracle.run(p, x.copy(), v.copy(), 1, first_half_kick=True)
    assert hits == 0
    dv = v1 - v
    expect = 0.5 * p.dt * (p.charge / p.mass)[:, None] * E
    np.testing.assert_allclose(dv, expect, rtol=1e-12, atol=1e-15)
    # opposite directions for the two species in the same field
    assert np.all(np.sign(dv[ion] * E[ion]) >= 0) and np.all(np.sign(dv[~ion] * E[~ion]) <= 0)


def test_collisions_act_on_electrons_only():
    p, x, v, ion = _mixed(n=400, L=1, seed=10)
    p.dt, p.nu_coll, p.wall_rule = 0.05, 50.0, 1
    p.n_tilde = 1e9  # fields negligible: velocity changes come from collisions
    x1, v1, _, _, _ = oracle.run(p, x.copy(), v.copy(), 1, first_half_kick=True)
    turned = np.linalg.norm(v1 - v, axis=1) > 1e-6 * np.linalg.norm(v, axis=1)
    assert np.any(turned[~ion])
    assert not np.any(turned[ion])

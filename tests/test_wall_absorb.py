"""Pins of the absorbing wall rule (wall_rule = 2) of the oracle.

The paper's probe floats: electrons that reach it stay on it, and its surface
charge Q_S is homogeneous on the surface S (Sec. 2), entering the field as
Q_S / (4 pi eps0 r) (Sec. 3). North_star asks the walls to absorb or re-inject.
The rule (a reading; the paper simulates diffuse reflection, Sec. 4): a
particle that crosses r = 1 is absorbed and its charge joins Q_S; one that
crosses r_out leaves; either is replaced, under the same id, by a particle
entering through the outer wall from the bulk plasma, whose entering flux is a
flux-weighted Maxwellian (inward normal speed of density v exp(-v^2 / 2 s^2),
tangential components normal with deviation s, s = lambda_D omega_pe).
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2111_13072_gb300.inputs import maxwellian_shell


def _params(n, L=4, r_out=1.6, sigma_v=0.05, **kw):
    vsh = 4 * np.pi / 3 * (r_out ** 3 - 1)
    return oracle.Params(d=0.2, eps=4.0, r_out=r_out, n_tilde=n / vsh, n_ion=float(n), L=L,
                         wall_rule=2, sigma_v=sigma_v, **kw)


def test_injection_is_the_flux_weighted_maxwellian():
    """Normal speeds follow the Rayleigh law of the crossing flux, the
    tangential components the Maxwellian, the entry points are isotropic on the
    outer sphere and the particles start inside, moving inwards."""
    s = 0.07
    p = _params(1000, sigma_v=s, dt=0.05)
    n = 200000
    x, v = oracle.inject(p, np.arange(n), step=7)
    r = np.linalg.norm(x, axis=1)
    nhat = x / r[:, None]
    vn = -np.einsum("ij,ij->i", v, nhat)
    assert np.all(vn > 0) and np.all(r < p.r_out) and np.all(r >= 1.0)
    # flux-weighted normal speed: CDF 1 - exp(-v^2 / (2 s^2))
    assert stats.kstest(vn, lambda t: 1 - np.exp(-t * t / (2 * s * s))).pvalue > 1e-3
    # the time since crossing is uniform over the step: r_out - r = u dt v_n
    u = (p.r_out - r) / (p.dt * vn)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # tangential components: normal, deviation s, independent of each other
    vt = v + vn[:, None] * nhat
    # a fixed tangent frame per point is arbitrary, so test the magnitude: the
    # tangential speed of two N(0, s^2) components is Rayleigh too
    vt_mag = np.linalg.norm(vt, axis=1)
    assert stats.kstest(vt_mag, lambda t: 1 - np.exp(-t * t / (2 * s * s))).pvalue > 1e-3
    assert np.max(np.abs(np.einsum("ij,ij->i", vt, nhat))) < 1e-12
    # isotropic entry points: mean 0, second moments 1/3
    assert np.all(np.abs(nhat.mean(axis=0)) < 5 / np.sqrt(3 * n))
    np.testing.assert_allclose((nhat ** 2).mean(axis=0), 1 / 3, atol=5 * np.sqrt(4 / 45 / n))
    # counter-based: the same (id, step) draws the same particle, another step not
    x2, v2 = oracle.inject(p, np.arange(10), step=7)
    np.testing.assert_array_equal(x2, x[:10])
    x3, _ = oracle.inject(p, np.arange(10), step=8)
    assert np.all(np.abs(x3 - x[:10]).max(axis=1) > 0)


def test_absorbed_charge_joins_the_surface_charge():
    """Every electron absorbed at the probe lowers Q_S by one super-particle
    charge; the particle count stays N and every particle stays in the domain."""
    n = 3000
    x, v = maxwellian_shell(n, 1.6, 0.08, seed=4)
    p = _params(n, sigma_v=0.08, dt=0.1, drive_kind=2, q_s=3.0)
    xo, vo, q, u, hits, q_s, nabs = oracle.run(p, x, v, 6, surface=True)
    assert nabs > 10 and hits > nabs  # some at the probe, more at the outer wall
    assert q_s == 3.0 - nabs
    r = np.linalg.norm(xo, axis=1)
    assert np.all((r >= 1.0) & (r <= p.r_out))


def test_surface_charge_enters_the_following_steps():
    """A run of 4 steps equals a run of 2 steps continued for 2 more with Q_S
    set to the value the first part accrued (the field of step n feels the
    charge absorbed in the steps before it)."""
    n = 2000
    x, v = maxwellian_shell(n, 1.6, 0.08, seed=9)
    p = _params(n, sigma_v=0.08, dt=0.1, drive_kind=2)
    xa, va, qa, ua, ha, qsa, na = oracle.run(p, x, v, 4, surface=True)
    x1, v1, q1, u1, h1, qs1, n1 = oracle.run(p, x, v, 2, surface=True)
    assert n1 > 0
    p2 = _params(n, sigma_v=0.08, dt=0.1, drive_kind=2, q_s=qs1)
    x2, v2, q2, u2, h2, qs2, n2 = oracle.run(p2, x1, v1, 2, step0=2, first_half_kick=False, surface=True)
    np.testing.assert_array_equal(xa, x2)
    np.testing.assert_array_equal(va, v2)
    assert qsa == qs2 and na == n1 + n2
    # and the accrued charge changed the trajectory (its field pushes the
    # electrons off the probe)
    p0 = _params(n, sigma_v=0.08, dt=0.1, drive_kind=2)
    x0, v0, _, _, _ = oracle.run(p0, x1, v1, 2, step0=2, first_half_kick=False)
    assert np.max(np.abs(x0 - x2)) > 0


def test_surface_charge_field_is_gauss():
    """The field of Q_S alone is Q_S / (4 pi n~ r^2) r^ (Sec. 3: Q_S/(4 pi eps0 r))."""
    p = _params(1, L=2, q_s=-7.0)
    p.n_ion = 0.0
    x = np.array([[0.3, -1.1, 0.9]])
    E = oracle.field_scan(p, x)
    r = np.linalg.norm(x)
    np.testing.assert_allclose(E[0], -7.0 / (4 * np.pi * p.n_tilde * r ** 3) * x[0], rtol=1e-13)


def test_no_wall_contact_means_no_difference():
    """Without wall contacts the rule changes nothing."""
    x, v = maxwellian_shell(600, 2.0, 1e-4, seed=2)
    keep = np.abs(np.linalg.norm(x, axis=1) - 1.5) < 0.4  # away from both walls
    x, v = x[keep], v[keep]
    n = len(x)
    p2 = _params(n, r_out=2.0, sigma_v=1e-4, dt=0.05, drive_kind=2)
    p0 = _params(n, r_out=2.0, sigma_v=1e-4, dt=0.05, drive_kind=2)
    p0.wall_rule = 0
    a = oracle.run(p2, x, v, 2)
    b = oracle.run(p0, x, v, 2)
    assert a[4] == 0 and b[4] == 0
    np.testing.assert_array_equal(a[0], b[0])

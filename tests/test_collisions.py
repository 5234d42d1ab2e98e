"""Electron-neutral collisions (the addition the paper's Sec. 5 names; the
Drude model of Sec. 4 damps with the collision rate nu): the oracle's
collision operator pinned by what its definition fixes -- a constant rate
nu, isotropic elastic scattering -- on the CPU."""
import numpy as np
import pytest

import oracle


def _params(nu, dt=0.05, seed=11):
    return oracle.Params(d=0.2, eps=4.0, r_out=2.0, n_tilde=100.0, n_ion=0.0, L=1, dt=dt, seed=seed,
                         nu_coll=nu)


def test_threshold_is_the_collision_probability():
    for nu, dt in ((0.2, 0.05), (1.0, 0.01), (3.0, 0.05)):
        assert oracle.coll_threshold(nu, dt) == int(np.floor((1.0 - np.exp(-nu * dt)) * 2 ** 24))
    assert oracle.coll_threshold(0.0, 0.05) == 0


def test_collisions_keep_the_speed_and_have_the_rate():
    n = 200000
    rng = np.random.default_rng(1)
    v = rng.standard_normal((n, 3))
    p = _params(2.0)
    P = 1.0 - np.exp(-2.0 * 0.05)
    v1, c = oracle.collisions(p, v, step=5)
    assert np.allclose(np.linalg.norm(v1, axis=1), np.linalg.norm(v, axis=1), rtol=1e-14)
    moved = np.any(v1 != v, axis=1)
    assert moved.sum() == c
    assert abs(c / n - P) < 5 * np.sqrt(P * (1 - P) / n)
    # the same step and seed draw the same numbers; another step others
    v2, c2 = oracle.collisions(p, v, step=5)
    np.testing.assert_array_equal(v1, v2)
    v3, _ = oracle.collisions(p, v, step=6)
    assert np.any(v3 != v1)


def test_scattering_is_isotropic():
    n = 200000
    v = np.tile([0.0, 0.0, 1.0], (n, 1))
    p = _params(1e6)  # P = 1 to within 2^-24: every particle scatters
    v1, c = oracle.collisions(p, v, step=0)
    assert c == n
    s = 4.0 / np.sqrt(n)
    assert np.all(np.abs(v1.mean(axis=0)) < 4 * np.sqrt(1 / 3) / np.sqrt(n))
    np.testing.assert_allclose((v1 ** 2).mean(axis=0), 1.0 / 3.0, atol=s)


def test_mean_velocity_relaxes_at_the_rate_nu():
    """A beam v = (1, 0, 0) under the collision operator alone: every collision
    leaves a direction of zero mean, so <v_x> after k steps is (1 - P)^k,
    = e^{-nu t} (the Drude momentum relaxation)."""
    n = 100000
    nu, dt = 1.5, 0.05
    p = _params(nu, dt)
    v = np.tile([1.0, 0.0, 0.0], (n, 1))
    P = oracle.coll_threshold(nu, dt) / 2 ** 24
    for k in range(1, 41):
        v, _ = oracle.collisions(p, v, step=k)
        if k % 10 == 0:
            expect = (1.0 - P) ** k
            assert abs(v[:, 0].mean() - expect) < 5 / np.sqrt(n)
            assert (1.0 - P) ** k == pytest.approx(np.exp(-nu * dt * k), rel=1e-6)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, rtol=1e-14)


def test_no_collisions_at_zero_rate():
    rng = np.random.default_rng(2)
    v = rng.standard_normal((1000, 3))
    v1, c = oracle.collisions(_params(0.0), v, step=3)
    assert c == 0
    np.testing.assert_array_equal(v1, v)

"""Pins of the oracle's Q_diff (Sec. 3 and Sec. 4) against the electrode charges
themselves.

The paper defines the response as Q_diff = (Q_1 - Q_2)/2 (Sec. 3), where Q_n is
the charge on electrode n from Gauss's law, Q_n = -int eps0 eps_r grad(Phi).df
over the electrode surface, and then writes the particle part as
Q_diff = -(1/n~) sum_i q_i Psi_anti(x_i) (Sec. 4). These tests compute Q_1 and
Q_2 without Psi_anti: by integrating the surface charge that each particle
induces on the two hemispheres of the electrode (R_E = 1 - d, the upper
hemisphere z > 0 is electrode 1) with a tensor quadrature on the sphere, and
compare (Q_1 - Q_2)/(2 n~) with the oracle's orc_qdiff. That fixes the sign,
the factor 1/2, the 1/n~ weight and the coefficients c_l' b^P_l of Psi_anti.

* eps = 1: the electrode is a grounded sphere in vacuum and the induced charge
  density is Kelvin's, sigma = -q (r^2 - a^2) / (4 pi a |x - a s|^3) (App. A,
  the mirror solution), a closed form with no series at all.
* eps = 4: the field at the electrode surface comes from the Green's function
  inside the dielectric, R^(d,p)_l = g_l (r_<^l / r_>^{l+1} - R_E^{2l+1} /
  (r r')^{l+1}) (Sec. 3), with g_l pinned separately by the interface
  conditions (test_oracle_pins). Its radial derivative at r = R_E is summed with
  Legendre polynomials of the angle between the surface point and the particle
  and integrated over each hemisphere; the permittivity enters through
  Gauss's law.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle


def _hemisphere_nodes(a, upper, nt=72, nphi=144):
    """Points and weights (area elements) of a tensor rule on one hemisphere of
    the sphere of radius a: Gauss-Legendre in cos(theta) on (0, 1) or (-1, 0),
    the periodic trapezoid rule in phi."""
    xg, wg = np.polynomial.legendre.leggauss(nt)
    ct = 0.5 * (xg + 1.0) if upper else 0.5 * (xg - 1.0)
    wct = 0.5 * wg
    phi = 2 * np.pi * np.arange(nphi) / nphi
    wphi = np.full(nphi, 2 * np.pi / nphi)
    CT, PH = np.meshgrid(ct, phi, indexing="ij")
    ST = np.sqrt(1.0 - CT * CT)
    s = np.stack([ST * np.cos(PH), ST * np.sin(PH), CT], axis=-1).reshape(-1, 3)  # unit normals
    w = (wct[:, None] * wphi[None, :]).reshape(-1) * a * a
    return s, w


def _particles(n, rmin, rmax, seed):
    rng = np.random.default_rng(seed)
    r = rng.uniform(rmin, rmax, n)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * r[:, None]


def _kelvin_charge(xk, q, a, s, w):
    """Charge induced on the surface patch (s, w) of a grounded sphere of radius
    a by a point charge q at xk (|xk| > a): integral of Kelvin's density."""
    r2 = float(xk @ xk)
    dist = np.linalg.norm(xk[None, :] - a * s, axis=1)
    sigma = -q * (r2 - a * a) / (4 * np.pi * a * dist ** 3)
    return float(np.sum(sigma * w))


def test_kelvin_quadrature_total_is_image_charge():
    """The rule integrates Kelvin's density to the image charge -q a / r (the
    quadrature itself is checked before it is used as a pin)."""
    a = 0.8
    up = _hemisphere_nodes(a, True)
    lo = _hemisphere_nodes(a, False)
    for xk in _particles(5, 1.3, 3.0, 11):
        tot = _kelvin_charge(xk, -1.0, a, *up) + _kelvin_charge(xk, -1.0, a, *lo)
        assert tot == pytest.approx(a / np.linalg.norm(xk), rel=1e-12)


@pytest.mark.parametrize("d", [0.2, 0.25])
def test_qdiff_equals_half_electrode_charge_difference_kelvin(d):
    """eps = 1: (Q_1 - Q_2)/(2 n~) from Kelvin's induced charge equals orc_qdiff."""
    a = 1.0 - d
    n_tilde = 123.4
    x = _particles(9, 1.6, 3.0, 3)
    p = oracle.Params(d=d, eps=1.0, r_out=3.5, n_tilde=n_tilde, n_ion=9.0, L=40)
    up = _hemisphere_nodes(a, True)
    lo = _hemisphere_nodes(a, False)
    q = -1.0  # electrons
    ref = sum(0.5 * (_kelvin_charge(xk, q, a, *up) - _kelvin_charge(xk, q, a, *lo)) for xk in x) / n_tilde
    got = oracle.qdiff(p, x)
    assert got == pytest.approx(ref, rel=1e-10)
    # one electron above the equator draws positive charge to electrode 1
    # (sigma = -q ... > 0), so Q_diff > 0
    xz = np.array([[0.1, 0.2, 2.0]])
    assert oracle.qdiff(p, xz) > 0.0


@pytest.mark.parametrize("eps,d", [(4.0, 0.2), (2.5, 0.25)])
def test_qdiff_from_gauss_law_in_the_dielectric(eps, d):
    """eps != 1: Q_n = -eps int_{E_n} dPhi/dr dA with Phi = q G (the Green's
    function inside the dielectric, g_l of App. A) equals, as (Q_1 - Q_2)/(2 n~),
    the oracle's -(1/n~) sum q Psi_anti."""
    RE = 1.0 - d
    Lser = 40
    g = oracle.coeffs(Lser, d, eps)["g"]
    n_tilde = 57.0
    x = _particles(7, 1.5, 2.8, 5)
    p = oracle.Params(d=d, eps=eps, r_out=3.0, n_tilde=n_tilde, n_ion=7.0, L=Lser)
    up = _hemisphere_nodes(RE, True)
    lo = _hemisphere_nodes(RE, False)
    ls = np.arange(Lser + 1)
    q = -1.0

    def charge(xk, s, w):
        rp = np.linalg.norm(xk)
        cg = s @ (xk / rp)  # cos of the angle between surface point and particle
        P = np.stack([eval_legendre(l, cg) for l in ls])  # [l][node]
        # d/dr of g_l (r^l / r'^{l+1} - RE^{2l+1} / (r r')^{l+1}) at r = RE
        dR = g * (2 * ls + 1) * RE ** (ls - 1.0) / rp ** (ls + 1.0)
        dG = ((dR * (2 * ls + 1) / (4 * np.pi))[:, None] * P).sum(axis=0)
        return float(-eps * q * np.sum(dG * w))

    ref = sum(0.5 * (charge(xk, *up) - charge(xk, *lo)) for xk in x) / n_tilde
    got = oracle.qdiff(p, x)
    assert got == pytest.approx(ref, rel=1e-9)
    # the two electrodes together hold the l = 0 part only: -q eps g_0 RE / r'
    # summed (Gauss's law for the whole sphere)
    tot = sum(charge(xk, *up) + charge(xk, *lo) for xk in x)
    exp_tot = sum(-q * eps * g[0] * RE / np.linalg.norm(xk) for xk in x)
    assert tot == pytest.approx(exp_tot, rel=1e-11)

"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
interface conditions the coefficients come from (App. A, Sec. 3), the Kelvin
mirror solution of the grounded sphere (App. A, the d = 0 / eps = 1 limit),
Legendre integrals of the hemisphere step, the dipole kernel printed in Sec. 3,
published random-number vectors, brute force against the radius-ordered scan,
and the invariants of the Hamiltonian dynamics (Sec. 2).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2111_13072_gb300.inputs import maxwellian_shell

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _shell_params(n, L, r_out=2.3, d=0.2, eps=4.0, **kw):
    vsh = 4 * np.pi / 3 * (r_out ** 3 - 1)
    return oracle.Params(d=d, eps=eps, r_out=r_out, n_tilde=n / vsh, n_ion=float(n), L=L, **kw)


# ---------------------------------------------------------------- coefficients
@pytest.mark.parametrize("l", [0, 1, 2, 5, 12])
@pytest.mark.parametrize("eps,d", [(4.0, 0.2), (1.0, 0.25), (2.5, 0.5), (10.0, 0.05)])
def test_radial_green_from_interface_conditions(l, eps, d):
    """Solve the radial equation of App. A directly (continuity of R_l and of
    eps dR_l/dr at r = R, R_l(R_E) = 0, decay, unit jump at r') and compare with
    R^(p,p)_l = (r_<^l/r_>^{l+1} - f_l/(r r')^{l+1})/(2l+1) and with
    R^(d,p)_l = g_l (r^l/r'^{l+1} - R_E^{2l+1}/(r r')^{l+1})."""
    c = oracle.coeffs(max(l, 1), d, eps)
    RE = 1.0 - d
    x = RE ** (2 * l + 1)
    rp = 1.7
    # unknowns: D (dielectric), A, B (1 < r < r'), C (r > r')
    M = np.array([
        [1 - x, -1.0, -1.0, 0.0],
        [eps * (l + (l + 1) * x), -l, (l + 1), 0.0],
        [0.0, rp ** l, rp ** (-(l + 1)), -rp ** (-(l + 1))],
        [0.0, -l * rp ** (l + 1), (l + 1) * rp ** (-l), -(l + 1) * rp ** (-l)],
    ])
    rhs = np.array([0.0, 0.0, 0.0, -1.0])
    D, A, B, C = np.linalg.solve(M, rhs)
    f, g = c["f"][l], c["g"][l]
    for r in (1.0, 1.3, 1.69):
        num = A * r ** l + B * r ** (-(l + 1))
        ref = (r ** l / rp ** (l + 1) - f / (r * rp) ** (l + 1)) / (2 * l + 1)
        assert num == pytest.approx(ref, rel=1e-12, abs=1e-15)
    for r in (2.0, 4.0):
        num = C * r ** (-(l + 1))
        ref = (rp ** l / r ** (l + 1) - f / (r * rp) ** (l + 1)) / (2 * l + 1)
        assert num == pytest.approx(ref, rel=1e-12, abs=1e-15)
    for r in (RE + 0.3 * d, RE + 0.9 * d):
        num = D * (r ** l - x * r ** (-(l + 1)))
        ref = g * (r ** l / rp ** (l + 1) - x / (r * rp) ** (l + 1))
        assert num == pytest.approx(ref, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("l", [0, 1, 3, 7, 15])
@pytest.mark.parametrize("eps,d", [(4.0, 0.2), (1.0, 0.3), (7.0, 0.5)])
def test_characteristic_function_coefficients(l, eps, d):
    """psi_l(R_E) = 1, psi_l and eps dpsi_l/dr continuous at R (Sec. 3)."""
    c = oracle.coeffs(max(l, 1), d, eps)
    RE = 1.0 - d
    M = np.array([[RE ** l, RE ** (-(l + 1)), 0.0],
                  [1.0, 1.0, -1.0],
                  [eps * l, -eps * (l + 1), (l + 1)]])
    a, b, bp = np.linalg.solve(M, [1.0, 0.0, 0.0])
    assert c["aD"][l] == pytest.approx(a, rel=1e-12, abs=1e-15)
    assert c["bD"][l] == pytest.approx(b, rel=1e-12, abs=1e-15)
    assert c["bP"][l] == pytest.approx(bp, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("eps,d", [(4.0, 0.2), (1.0, 0.2), (3.0, 0.7)])
def test_floating_potential_cancels_monopole_image(eps, d):
    """The Psi_sym coefficient for r >= R (Sec. 3) equals f_0 (App. A), so the
    modified Green's function keeps 1/(4 pi r_>) as its l = 0 term (Sec. 3)."""
    c = oracle.coeffs(1, d, eps)
    psi_sym = (1 - d) * eps / (d + eps - d * eps)
    assert c["f"][0] == pytest.approx(psi_sym, rel=1e-14)
    assert c["bP"][0] == pytest.approx(psi_sym, rel=1e-14)


def test_psi_anti_legendre_coefficients():
    """c_l' against the printed rationals and against the Legendre projection
    of the hemisphere step +1/2 (upper) / -1/2 (lower)."""
    from fractions import Fraction
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "psi_anti_coeffs.txt"))
            if ln.strip() and not ln.startswith("#")]
    L = 31
    c = oracle.coeffs(L, 0.2, 4.0)
    cprime = np.where(c["bP"] != 0, c["canti"] / c["bP"], 0.0)
    for lp, l, frac in rows:
        assert cprime[int(l)] == pytest.approx(float(Fraction(frac)), rel=1e-14)
    xg, wg = np.polynomial.legendre.leggauss(64)
    xs, ws = 0.5 * (xg + 1.0), 0.5 * wg  # nodes on [0, 1]
    for l in range(1, L + 1):
        Pl = np.polynomial.legendre.Legendre.basis(l)(xs)
        proj = (2 * l + 1) / 2.0 * np.sum(ws * Pl) if l % 2 == 1 else 0.0
        assert cprime[l] == pytest.approx(proj, rel=1e-12, abs=1e-14)


# ---------------------------------------------------------------- Green's function
@pytest.mark.parametrize("x,xs", [
    ([0.3, -1.1, 2.7], [0.9, 0.5, -0.4]),
    ([1.05, 0.2, -0.1], [-1.3, 1.6, 1.2]),
    ([0.0, 0.0, 4.0], [0.7, 0.0, 0.8]),
])
def test_kelvin_limit(x, xs):
    """eps = 1: the dielectric is vacuum and G is the Kelvin mirror solution of a
    grounded sphere of radius R_E (App. A). G~ adds R_E/(4 pi r r') (floating
    potential, Sec. 3). With r_</r_> <= 0.5 and L = 60 the series tail < 1e-12."""
    d = 0.2
    RE = 1 - d
    p = _shell_params(10, 60, d=d, eps=1.0)
    x = np.array(x, float)
    xs = np.array(xs, float)
    r, rs = np.linalg.norm(x), np.linalg.norm(xs)
    assert min(r, rs) / max(r, rs) <= 0.5
    ximg = (RE ** 2 / rs ** 2) * xs
    G_ref = (1 / np.linalg.norm(x - xs) - RE / (rs * np.linalg.norm(x - ximg)) + RE / (r * rs)) / (4 * np.pi)
    dG_ref = (-(x - xs) / np.linalg.norm(x - xs) ** 3
              + RE / rs * (x - ximg) / np.linalg.norm(x - ximg) ** 3
              - RE * x / (r ** 3 * rs)) / (4 * np.pi)
    G, dG = oracle.green(p, x, xs)
    assert G == pytest.approx(G_ref, rel=1e-11)
    np.testing.assert_allclose(dG, dG_ref, rtol=1e-10, atol=1e-12 * np.linalg.norm(dG_ref))


def test_dipole_kernel_printed_in_paper():
    """m0_only with L = 1 is the truncated kernel printed at the end of Sec. 3,
    (1/4pi)[1/r_> + (r_</r_>^2 - f_1/(r^2 r'^2)) cos t cos t'] (reading: the
    second 1/(4 pi) printed inside the bracket is a typo)."""
    d, eps = 0.25, 4.0
    f1 = oracle.coeffs(1, d, eps)["f"][1]
    p = _shell_params(10, 1, d=d, eps=eps, m0_only=1)
    rng = np.random.default_rng(3)
    for _ in range(20):
        x, xs = rng.normal(size=3) * 1.5, rng.normal(size=3) * 1.5
        x *= max(1.0, 1.01 / np.linalg.norm(x))
        xs *= max(1.0, 1.01 / np.linalg.norm(xs))
        r, rs = np.linalg.norm(x), np.linalg.norm(xs)
        rl, rg = min(r, rs), max(r, rs)
        ref = (1 / rg + (rl / rg ** 2 - f1 / (r * r * rs * rs)) * (x[2] / r) * (xs[2] / rs)) / (4 * np.pi)
        G, _ = oracle.green(p, x, xs)
        assert G == pytest.approx(ref, rel=1e-13)


# ---------------------------------------------------------------- evaluators
@pytest.mark.parametrize("n,L,m0,si,qs,u", [
    (257, 6, 0, 0, 0.0, 0.0),
    (301, 8, 0, 1, 3.0, 0.02),
    (64, 3, 1, 0, -2.0, 0.5),
    (97, 12, 0, 0, 0.0, 0.01),
    (2, 5, 0, 1, 0.0, 0.0),
])
def test_scan_matches_brute_force(n, L, m0, si, qs, u):
    x, _ = maxwellian_shell(n, 2.3, 0.05, seed=n)
    p = _shell_params(n, L, m0_only=m0, self_image=si, q_s=qs)
    Eb = oracle.field_brute(p, x, u=u)
    Es = oracle.field_scan(p, x, u=u)
    assert np.linalg.norm(Es - Eb) <= 1e-12 * np.linalg.norm(Eb)
    sample = np.array([0, n // 2, n - 1])
    np.testing.assert_array_equal(oracle.field_brute(p, x, u=u, sample=sample), Eb[sample])


@pytest.mark.parametrize("L,r_out", [(16, 5.2), (24, 3.5)])
def test_scan_matches_brute_force_per_particle_wide_shell(L, r_out):
    """A wide shell at a high degree: the outermost particles' suffix moments
    are about (1 / r_out)^(l+1) of the totals (5^-17 here), so a suffix formed
    as total minus prefix would lose five digits; summed from the outside in,
    the scan matches the pair sum for every particle to 1e-11 (relative to the
    particle's own field)."""
    n = 1200
    x, _ = maxwellian_shell(n, r_out, 0.05, seed=7)
    p = _shell_params(n, L, r_out=r_out, self_image=1)
    Eb = oracle.field_brute(p, x)
    Es = oracle.field_scan(p, x)
    err = np.linalg.norm(Es - Eb, axis=1) / np.linalg.norm(Eb, axis=1)
    assert err.max() < 1e-11, err.max()


def test_neutral_shell_monopole_cancels():
    """Uniform electrons over the same shell as the uniform ion background:
    the l = 0 fields cancel up to sqrt(N) fluctuations (a wrong sign or scale of
    the ion term would leave a field of order N/(4 pi n~))."""
    n = 4000
    x, _ = maxwellian_shell(n, 2.0, 0.0, seed=11)
    p = _shell_params(n, 0, r_out=2.0)
    E = oracle.field_scan(p, x)
    scale = n / (4 * np.pi * p.n_tilde)
    rms = np.sqrt(np.mean(np.sum(E ** 2, axis=1)))
    assert rms < 4.0 * np.sqrt(n) / (4 * np.pi * p.n_tilde)
    assert rms < 0.05 * scale


# ---------------------------------------------------------------- dynamics
def _quiet_setup(n=48, L=4, seed=5):
    x, v = maxwellian_shell(n, 2.6, 0.02, seed=seed, r_in=1.4)
    p = oracle.Params(d=0.2, eps=4.0, r_out=3.5, n_tilde=10.0, n_ion=float(n), L=L, wall_rule=1,
                      drive_kind=2)
    return p, x, v


@pytest.mark.parametrize("si,qs,u", [(0, 0.0, 0.0), (1, 0.7, 0.3), (0, -1.5, 0.05)])
def test_force_is_energy_gradient(si, qs, u):
    """The field of every term (pairs through G~, self image, ion background,
    Q_S, drive) is minus the gradient of the Hamiltonian of Sec. 2 divided by
    q = -1, checked by central differences of H."""
    p, x, v = _quiet_setup()
    p.self_image, p.q_s = si, qs
    E = oracle.field_brute(p, x, u=u)
    h = 1e-6
    for k in (0, 7, 30, 47):
        g = np.zeros(3)
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            g[c] = (oracle.energy(p, xp, v, u=u) - oracle.energy(p, xm, v, u=u)) / (2 * h)
        np.testing.assert_allclose(E[k], g, rtol=1e-6, atol=1e-9)


def _sync_energy(p, x, vhalf, dt):
    E = oracle.field_scan(p, x)
    return oracle.energy(p, x, vhalf - 0.5 * dt * E)


def test_energy_conservation_drive_off():
    """Drive off, no wall hits: H of Sec. 2 stays constant to a small fraction
    of the kinetic energy exchanged. (The 1/r_> kernel has a kink wherever two
    radii cross, so the error does not follow the smooth-force dt^2 law.)"""
    p, x, v = _quiet_setup()
    dt = p.dt = 0.05
    H0 = oracle.energy(p, x, v)
    K0 = 0.5 * np.sum(v * v)
    worst, dK = 0.0, 0.0
    first = True
    for c in range(8):
        x, v, _, _, hits = oracle.run(p, x, v, 10, step0=c * 10, first_half_kick=first)
        first = False
        assert hits == 0
        worst = max(worst, abs(_sync_energy(p, x, v, dt) - H0))
        E = oracle.field_scan(p, x)
        vs = v - 0.5 * dt * E
        dK = max(dK, abs(0.5 * np.sum(vs * vs) - K0))
    assert worst < 1e-4 * abs(H0)
    assert worst < 0.01 * dK


def test_angular_momentum_conservation():
    """G~ is rotation invariant and Psi_anti is axisymmetric: with the drive on,
    L_z = sum x v_y - y v_x is conserved to rounding; with the drive off, all of L."""
    p, x, v = _quiet_setup(n=40, L=6, seed=9)
    for drive, comps in ((0, [2]), (2, [0, 1, 2])):
        p.drive_kind = drive
        p.v_hat = 0.05
        p.sigma, p.t0 = 0.5, 1.0
        L0 = np.sum(np.cross(x, v), axis=0)
        x1, v1, q, u, hits = oracle.run(p, x, v, 60)
        assert hits == 0
        L1 = np.sum(np.cross(x1, v1), axis=0)
        scale = np.sum(np.linalg.norm(x, axis=1) * np.linalg.norm(v, axis=1))
        for c in comps:
            assert abs(L1[c] - L0[c]) < 1e-12 * scale
        if drive == 0:
            assert np.max(np.abs(u)) > 0.04  # the pulse did act


def test_philox_known_answers():
    for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        h = [int(t, 16) for t in ln.split()]
        out = oracle.philox4x32_10(h[0:4], h[4:6])
        assert list(out) == h[6:10]


def test_diffuse_wall_keeps_speed_and_points_inward():
    p = _shell_params(200, 2, r_out=2.0, wall_rule=0, drive_kind=2)
    p.n_tilde = 1e12  # negligible fields: only the walls act
    rng = np.random.default_rng(4)
    n = 200
    dirs = rng.normal(size=(n, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    inner = np.arange(n) < n // 2
    r = np.where(inner, 1.0005, 1.9995)
    x = dirs * r[:, None]
    v = -dirs * np.where(inner, 0.1, -0.1)[:, None]  # moving into the walls
    x1, v1, _, _, hits = oracle.run(p, x, v, 1, first_half_kick=False)
    assert hits == n
    np.testing.assert_allclose(np.linalg.norm(v1, axis=1), 0.1, rtol=1e-10)
    rad = np.sum(v1 * x1, axis=1) / np.linalg.norm(x1, axis=1)
    assert np.all(rad[inner] > 0) and np.all(rad[~inner] < 0)
    rr = np.linalg.norm(x1, axis=1)
    assert np.all(rr >= 1.0) and np.all(rr <= 2.0)
    # isotropic over the hemisphere: cos of the angle to the normal is uniform
    cosang = np.abs(rad) / 0.1
    assert abs(np.mean(cosang) - 0.5) < 0.06


def test_spectrum_of_damped_sine():
    """Y = i w Q^/U^ of an impulse response a e^{-bt} sin(ct) has its Re Y peak
    at ~c with full width ~2b (Lorentzian limit); the fit recovers (a, b, c)."""
    dt, ns = 0.05, 8000
    a, b, c = 1.089, 0.06317, 0.5352  # the fit printed in Sec. 4
    t = dt * np.arange(ns)
    q = a * np.exp(-b * t) * np.sin(c * t)
    u = np.zeros(ns)
    u[0] = 1.0 / (0.5 * dt)  # unit impulse with the half first kick
    om, Y, wr, dw = oracle.spectrum(q, u, dt, 4000, 2.0)
    assert wr == pytest.approx(np.sqrt(c * c + b * b), rel=0.01)
    assert dw == pytest.approx(2 * b, rel=0.05)
    fit = oracle.fit_damped_sine(q, dt, 0.0, wr, dw / 2)
    np.testing.assert_allclose(fit[:3], [a, b, c], rtol=1e-6)

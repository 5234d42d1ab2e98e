"""Drude fit and temperature diagnostic (Sec. 4), on the CPU: the library's
host-side fit (through the C ABI; it needs no GPU) and the oracle's fit,
each pinned by closed forms and by the values the paper prints."""
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _golden():
    vals, sweep = {}, []
    for line in open(os.path.join(ROOT, "tests", "golden", "drude_paper_values.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "sweep":
            sweep.append((float(line[1]), float(line[2])))
        else:
            vals[line[0]] = float(line[1])
    return vals, sweep


@pytest.fixture(scope="module")
def imrp():
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


def _model(omega, C, eta, nu):
    """i w C eta^2 / (eta^2 - w^2 + i w nu), written out independently of both fits."""
    return 1j * omega * C * eta ** 2 / (eta ** 2 - omega ** 2 + 1j * omega * nu)


CASES = [(0.8, 0.55, 0.126), (2.5, 0.9, 0.05), (0.3, 0.4, 0.3)]


def test_fwhm_of_drude_real_part_equals_nu():
    """Re Y_D = C w^2 eta^2 nu / ((eta^2 - w^2)^2 + w^2 nu^2) peaks at eta, and its
    half maximum lies where eta^2 - w^2 = +-w nu, so its full width is exactly nu."""
    w = np.linspace(1e-4, 2.0, 400001)
    for C, eta, nu in CASES:
        w_res, dw = oracle.peak_and_fwhm(w, _model(w, C, eta, nu).real)
        assert abs(w_res - eta) < 1e-6
        assert abs(dw - nu) < 1e-6


@pytest.mark.parametrize("C,eta,nu", CASES)
def test_fits_recover_an_exact_drude_admittance(imrp, C, eta, nu):
    w = np.linspace(0.002, 1.5, 1500)
    Y = _model(w, C, eta, nu)
    for fit in (oracle.drude_fit(w, Y, 0.0, 1.5), imrp.drude_fit(w, Y.real, Y.imag, 0.0, 1.5)):
        assert fit[0] == pytest.approx(C, rel=1e-8)
        assert fit[1] == pytest.approx(eta, rel=1e-8)
        assert fit[2] == pytest.approx(nu, rel=1e-8)
        assert fit[3] < 1e-8


def test_paper_damped_sine_is_a_drude_resonance(imrp):
    """The paper's fitted signal f(t) = a e^{-bt} sin(ct) after a unit kick has the
    admittance i w a c / ((b + i w)^2 + c^2), a Drude dipole term with nu = 2b,
    eta = sqrt(b^2 + c^2), C = a c / eta^2: both fits return these (the paper
    quotes the matched nu_eff = 0.128 against 2b = 0.126)."""
    g, _ = _golden()
    a, b, c = g["a"], g["b"], g["c"]
    w = np.linspace(0.001, 1.0, 2000)
    Y = 1j * w * a * c / ((b + 1j * w) ** 2 + c ** 2)
    eta = np.hypot(b, c)
    for fit in (oracle.drude_fit(w, Y, 0.0, 1.0), imrp.drude_fit(w, Y.real, Y.imag, 0.0, 1.0)):
        assert fit[2] == pytest.approx(2 * b, rel=1e-8)
        assert fit[1] == pytest.approx(eta, rel=1e-8)
        assert fit[0] == pytest.approx(a * c / eta ** 2, rel=1e-8)


def test_fits_agree_on_a_noisy_admittance(imrp):
    """Away from an exact model both minimise the same integral: same optimum."""
    rng = np.random.default_rng(7)
    w = np.linspace(0.01, 1.2, 700)
    Y = _model(w, 1.3, 0.62, 0.11) + 0.02 * (rng.standard_normal(w.size) + 1j * rng.standard_normal(w.size))
    Y += 0.05 * w ** 2  # a smooth background the model cannot follow
    o = oracle.drude_fit(w, Y, 0.0, 1.0)
    c = imrp.drude_fit(w, Y.real, Y.imag, 0.0, 1.0)
    for k in range(3):
        assert c[k] == pytest.approx(o[k], rel=1e-6)
    assert c[3] == pytest.approx(o[3], rel=1e-6)


def test_temperature_diagnostic_reproduces_the_paper(imrp):
    """nu_eff = K lambda_D w_pe / R with the paper's sweep: K is 1.26 for each
    temperature and 1.264 on average, and inverting with K = 1.264 returns the
    temperatures within the rounding of the printed rates."""
    g, sweep = _golden()
    R, n = g["R_m"], g["n_e_m3"]
    Ks = []
    for T, nu in sweep:
        K = imrp.drude_k(nu, T, R, n)
        assert K == pytest.approx(oracle.drude_K(nu, T, R, n), rel=1e-12)
        assert K == pytest.approx(g["K_3eV"], abs=0.015)
        Ks.append(K)
        Te = imrp.drude_te(nu, g["K_sweep"], R, n)
        assert Te == pytest.approx(oracle.drude_Te(nu, g["K_sweep"], R, n), rel=1e-12)
        assert Te == pytest.approx(T, rel=0.015)
    assert np.mean(Ks) == pytest.approx(g["K_sweep"], abs=0.002)
    assert imrp.drude_k(0.128, 3.0, R, n) == pytest.approx(g["K_3eV"], abs=0.005)


def test_drude_fit_rejects_bad_input(imrp):
    w = np.linspace(0.1, 1.0, 10)
    y = _model(w, 1.0, 0.5, 0.1)
    with pytest.raises(imrp.IMRPError):
        imrp.drude_fit(w, y.real, y.imag, 2.0, 3.0)  # no point in the window
    with pytest.raises(imrp.IMRPError):
        imrp.drude_fit(w[::-1], y.real, y.imag, 0.0, 1.0)  # omega not increasing
    with pytest.raises(imrp.IMRPError):
        imrp.drude_k(-0.1, 3.0, 0.004, 1e15)


def test_damped_sine_fit_of_a_series(imrp):
    """The library's fit of a given series returns the paper's printed signal
    (Sec. 4) from its samples, as the oracle's fit does, within a time window."""
    g, _ = _golden()
    a, b, c = g["a"], g["b"], g["c"]
    dt = 0.01
    t = dt * np.arange(6000)
    q = a * np.exp(-b * t) * np.sin(c * t)
    q[t > 40.0] += 5.0  # outside the window: must not matter
    fit = imrp.fit_damped_sine(q, dt, 0.0, 40.0, 0.5, 0.05)
    np.testing.assert_allclose(fit[:3], [a, b, c], rtol=1e-9)
    assert min(fit[3], 2 * np.pi - fit[3]) < 1e-8
    fo = oracle.fit_damped_sine(q[t <= 40.0], dt, 0.0, 0.5, 0.05)
    np.testing.assert_allclose(fit[:3], fo[:3], rtol=1e-8)

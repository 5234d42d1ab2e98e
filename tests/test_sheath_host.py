"""The library's floating equilibrium (App. D; host code behind the C ABI, no
GPU) against the oracle's, its argument checks, and the radial-profile input
sampler. CPU only."""
import numpy as np
import pytest

from oracle import sheath as S
from paper_2111_13072_gb300.inputs import radial_profile_shell

ARGON = 39.948 * 1822.888486


@pytest.fixture(scope="module")
def imrp():
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


# (lambda_D / R, r_out, nodes): the paper's Fig. 5 case (3 eV, 1e15 m^-3, R = 4 mm),
# a thin sheath, a thick one on a coarse grid
CASES = [(0.10183, 10.0, 2049), (0.02, 4.0, 257), (0.3, 10.0, 101)]


@pytest.mark.parametrize("lam,r_out,n", CASES)
def test_sheath_solve_matches_oracle(imrp, lam, r_out, n):
    p = imrp.sheath_solve(lam, ARGON, r_out, n)
    o = S.equilibrium(lam, ARGON, r_out, n)
    assert p["rhat"] == pytest.approx(o["rhat"], rel=1e-9)
    assert p["psi_wall"] == pytest.approx(o["psi_wall"], rel=1e-9)
    assert p["q_s"] == pytest.approx(o["q_s"], rel=1e-8)
    assert abs(p["residual"]) < 1e-9
    np.testing.assert_allclose(p["r"], o["r"], rtol=1e-15)
    np.testing.assert_allclose(p["psi"], o["psi"], rtol=1e-8)
    np.testing.assert_allclose(p["dpsi"], o["dpsi"], rtol=1e-7, atol=1e-9 * abs(o["dpsi"][0]))
    for k in ("q_ion", "q_elec"):
        assert p[k][0] == 0.0
        np.testing.assert_allclose(p[k], o[k], rtol=0, atol=1e-9 * o[k][-1])


def test_sheath_solve_rejects_bad_arguments(imrp):
    for args in [(0.0, ARGON, 10.0, 9), (-0.1, ARGON, 10.0, 9), (0.1, 3.0, 10.0, 9),
                 (0.1, ARGON, 1.0, 9), (0.1, ARGON, 10.0, 1), (float("nan"), ARGON, 10.0, 9),
                 # Bohm radius outside the domain: a Debye length as large as the domain
                 (3.0, ARGON, 1.2, 9)]:
        with pytest.raises(imrp.IMRPError):
            imrp.sheath_solve(*args)


def test_radial_profile_sampler_follows_the_table():
    lam = 0.10183
    e = S.equilibrium(lam, ARGON, 10.0, 1025)
    n = 400000
    x, v = radial_profile_shell(n, e["r"], e["q_elec"], lam, seed=5)
    r = np.linalg.norm(x, axis=1)
    assert r.min() > 1.0 and r.max() < 10.0
    edges = np.array([1.0, 1.1, 1.3, 1.6, 2.0, 3.0, 5.0, 7.5, 10.0])
    counts = np.histogram(r, edges)[0]
    expect = np.diff(np.interp(edges, e["r"], e["q_elec"])) / e["q_elec"][-1] * n
    # multinomial counts: within 5 standard deviations
    assert np.all(np.abs(counts - expect) < 5 * np.sqrt(expect) + 1)
    # isotropic directions, thermal velocities of standard deviation lambda_D / R
    assert np.abs(np.mean(x / r[:, None], axis=0)).max() < 0.01
    assert np.std(v) == pytest.approx(lam, rel=0.01)

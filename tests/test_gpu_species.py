"""Mobile ions on the GPU path (imrp_set_species): the paper moves its ions as
super-particles like the electrons (Sec. 4). Ions of charge +1 and mass m_i
take part in the moments, the pair sums and the l = 0 inner charge with their
charge, and are pushed with their q/m. Field and steps against the oracle with
the same per-particle charges and masses (orc_field_params.charge / .mass,
pinned in tests/test_oracle_species.py)."""
import numpy as np
import pytest

import oracle
from paper_2111_13072_gb300.inputs import Workload, workload_state
from parity_metrics import TOL, check_field

pytestmark = pytest.mark.gpu

W = Workload("species", N=3000, l_max=8, T_e_eV=20.0, n_e_m3=1e15, drive_kind=1, V_volts=50.0)
M_ION = 100.0  # a light ion, so that it moves visibly in a few steps


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


def _state(n, n_e):
    x, v = workload_state(W, N=n)
    v = v.copy()
    v[n_e:] /= np.sqrt(M_ION)  # ions as hot as the electrons, so slower by sqrt(m_i / m_e)
    return x, v


def _oracle(p, n, n_e, bg, L):
    op = oracle.from_physical(W.R_E_m, W.R_D_m, W.eps_D, W.R_out_m, W.n_e_m3, W.T_e_eV, n, L, p.dt,
                              drive_kind=p.drive_kind, V_volts=p.V_volts, width_wpe=p.width_wpe,
                              wall_rule=p.wall_rule, self_image=p.self_image, seed=p.seed)
    vsh = 4 * np.pi / 3 * (op.r_out ** 3 - 1)
    op.n_tilde = n_e / vsh  # n~ counts the electrons
    op.n_ion = float(bg)
    op.charge = np.concatenate([-np.ones(n_e), np.ones(n - n_e)])
    op.mass = np.concatenate([np.ones(n_e), np.full(n - n_e, M_ION)])
    return op


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,n_e,L,si", [(3000, 2000, 8, 0), (3000, 2000, 16, 1), (900, 600, 4, 0)])
def test_field_and_steps_with_mobile_ions(imrp, prec, n, n_e, L, si):
    bg = n_e - (n - n_e)  # the immobile background makes up the rest of the neutralising ions
    x, v = _state(n, n_e)
    p = imrp.params_from_workload(W, N=n, precision=prec, l_max=L, self_image=si)
    op = _oracle(p, n, n_e, bg, L)
    with imrp.Sim(p) as sim:
        sim.set_species(n_e, 1.0, M_ION, bg)
        sim.load(x, v)
        info = sim.info()
        assert info.n_tilde == pytest.approx(op.n_tilde, rel=1e-12) and info.n_ion == bg
        E = sim.field()
        q, _ = sim.step(3)
        xg, vg = sim.particles()
    Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
    check_field(E, Eo, prec, f"ions n={n} L={L}")
    xo, vo, qo, _, hits = oracle.run(op, x, v, 3)
    dv_g, dv_o = vg - v, vo - v
    per = np.linalg.norm(dv_g - dv_o, axis=1) / (np.linalg.norm(dv_o, axis=1) + 1e-30)
    bad = per > 10 * TOL[prec]
    assert np.sum(bad) <= (0 if prec == 0 else 2), f"{np.sum(bad)} particles differ"
    ions = np.arange(n) >= n_e
    # the ions moved by their own, smaller q/m
    assert np.linalg.norm(dv_o[ions], axis=1).mean() < 0.5 * np.linalg.norm(dv_o[~ions], axis=1).mean()
    for sel in (ions, ~ions):
        good = sel & ~bad
        assert np.linalg.norm(dv_g[good] - dv_o[good]) / np.linalg.norm(dv_o[good]) < 10 * TOL[prec]
        assert np.linalg.norm(xg[good] - xo[good]) / np.linalg.norm(xo[good]) < TOL[prec]
    np.testing.assert_allclose(q, qo, rtol=10 * TOL[prec], atol=10 * TOL[prec] * np.max(np.abs(qo)))


@pytest.mark.parametrize("prec", [0, 1])
def test_species_without_ions_is_the_electron_path(imrp, prec):
    """All particles flagged electrons: the scanned inner charge is the sorted
    count exactly (integers in FP64), so field and steps are bit for bit the
    default path's; ion_charge = 0 switches the mode off again."""
    n = 2500
    x, v = workload_state(W, N=n)
    p = imrp.params_from_workload(W, N=n, precision=prec)
    with imrp.Sim(p) as a, imrp.Sim(p) as b:
        a.load(x, v)
        b.set_species(n, 1.0, M_ION, float(n))
        b.load(x, v)
        np.testing.assert_array_equal(a.field(), b.field())
        qa, _ = a.step(3)
        qb, _ = b.step(3)
        np.testing.assert_array_equal(qa, qb)
        np.testing.assert_array_equal(a.particles()[0], b.particles()[0])
        b.set_species(n, 0.0, 0.0, 0.0)
        np.testing.assert_array_equal(a.field(), b.field())


def test_species_rejects_bad_arguments(imrp):
    p = imrp.params_from_workload(W, N=100)
    with imrp.Sim(p) as sim:
        for args in ((0, 1.0, 10.0, 0.0), (50, -1.0, 10.0, 0.0), (50, 1.0, 0.0, 0.0), (101, 1.0, 10.0, 0.0),
                     (50, 1.0, 10.0, -1.0)):
            with pytest.raises(imrp.IMRPError):
                sim.set_species(*args)
    p2 = imrp.params_from_workload(W, N=100, wall_rule=2)
    with imrp.Sim(p2) as sim:
        with pytest.raises(imrp.IMRPError):
            sim.set_species(50, 1.0, 10.0, 0.0)

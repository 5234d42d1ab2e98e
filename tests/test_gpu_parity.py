"""GPU path (C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (stated by the method's precision contract): the field E at every
particle matches to 1e-5 relative (||dE|| / ||E|| over all particles) on the
FP64 path and to 1e-4 on the mixed path (FP32 state, harmonics and push with
FP64 carries). The inputs are float32-representable, so both paths and the
oracle start from identical states.
"""
import numpy as np
import pytest

import oracle
from paper_2111_13072_gb300.inputs import WORKLOADS, Workload, maxwellian_shell, workload_state

pytestmark = pytest.mark.gpu

from parity_metrics import P999, TOL, check_field


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available(), "these tests need the GPU"
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


def _pair(imrp, w: Workload, n, **over):
    """GPU params and oracle params of workload w with n particles."""
    p = imrp.params_from_workload(w, N=n, **{k: v for k, v in over.items() if k != "t0_wpe"})
    op = oracle.from_physical(w.R_E_m, w.R_D_m, w.eps_D, w.R_out_m, w.n_e_m3, w.T_e_eV, n,
                              p.l_max, p.dt, drive_kind=p.drive_kind, V_volts=p.V_volts,
                              width_wpe=p.width_wpe, wall_rule=p.wall_rule,
                              self_image=p.self_image, seed=p.seed, nu_coll=p.nu_coll)
    return p, op


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


BASE = WORKLOADS["fp64_n2e4_l8"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,L", [(1, 8), (2, 4), (31, 8), (32, 4), (33, 2), (1000, 1), (1024, 8),
                                 (1025, 8), (4103, 12), (8269, 8), (3001, 16), (1500, 24)])
def test_field_matches_oracle(imrp, prec, n, L):
    x, v = workload_state(BASE, N=n)
    p, op = _pair(imrp, BASE, n, precision=prec, l_max=L)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        E = sim.field()
    Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
    if n == 1:
        # a lone electron feels only the ions, its image is excluded: compare directly
        np.testing.assert_allclose(E, Eo, rtol=TOL[prec], atol=0)
    else:
        check_field(E, Eo, prec, f"n={n} L={L}")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,L", [(150000, 16), (100003, 24), (600001, 2), (250001, 16), (1300001, 2)])
def test_field_matches_oracle_every_particle_large(imrp, prec, n, L):
    """Every particle at sizes beyond one segment of the group scan (more than
    64 groups of 1024 particles: the multi-segment sums, the ticketed last-CTA
    scan and the segment bases all run), at the bench's degree and at the
    largest one, and beyond 2^19 particles (the sort's 9-bit top pass into 512
    buckets) at a low degree; the last two with at least twice as many tiles
    as the GPU holds resident warps (several waves of field CTAs). Against the
    oracle's scan evaluator."""
    x, v = workload_state(BASE, N=n)
    p, op = _pair(imrp, BASE, n, precision=prec, l_max=L, drive_kind=1, V_volts=50.0)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        E = sim.field()
    Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
    check_field(E, Eo, prec, f"n={n} L={L}")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("self_image,drive,V,qs", [(1, 1, 300.0, 0.0), (0, 1, 300.0, 0.0),
                                                   (1, 2, 1.0, 0.0)])
def test_field_terms(imrp, prec, self_image, drive, V, qs):
    """Self image on/off and a strong impulse drive (u_asy Psi_anti term)."""
    n = 2500
    x, v = workload_state(BASE, N=n)
    p, op = _pair(imrp, BASE, n, precision=prec, self_image=self_image, drive_kind=drive,
                  V_volts=V)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        E = sim.field()
    Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
    check_field(E, Eo, prec, f"self_image={self_image} drive={drive}")


@pytest.mark.parametrize("prec", [0, 1])
def test_steps_match_oracle(imrp, prec):
    """Three leapfrog steps with diffuse walls: velocity changes, positions,
    wall hits and Q_diff against the oracle's run."""
    n = 3000
    w = Workload("walls", N=n, l_max=8, T_e_eV=20.0, n_e_m3=1e15, drive_kind=1, V_volts=50.0)
    x, v = workload_state(w, N=n)
    p, op = _pair(imrp, w, n, precision=prec)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        q, u = sim.step(3)
        xg, vg = sim.particles()
    xo, vo, qo, uo, hits = oracle.run(op, x, v, 3)
    assert hits > 0
    np.testing.assert_allclose(u, uo, rtol=1e-12, atol=0)
    dv_g, dv_o = vg - v, vo - v
    per = np.linalg.norm(dv_g - dv_o, axis=1) / (np.linalg.norm(dv_o, axis=1) + 1e-30)
    bad = np.sum(per > 10 * TOL[prec])
    assert bad <= (0 if prec == 0 else 2), f"{bad} particles differ"
    good = per <= 10 * TOL[prec]
    assert _rel(dv_g[good], dv_o[good]) < TOL[prec] * 10
    assert _rel(xg[good], xo[good]) < TOL[prec]
    np.testing.assert_allclose(q, qo, rtol=10 * TOL[prec], atol=10 * TOL[prec] * np.max(np.abs(qo)))


@pytest.mark.parametrize("prec", [0, 1])
def test_collision_steps_match_oracle(imrp, prec):
    """Five steps with electron-neutral collisions (nu = 2: about 10 % of the
    particles scatter per step) and diffuse walls: the same particles scatter
    on both sides (the decision is an integer compare of the same Philox word),
    and velocities and positions agree."""
    n = 3000
    w = Workload("coll", N=n, l_max=8, T_e_eV=20.0, n_e_m3=1e15, drive_kind=1, V_volts=50.0)
    x, v = workload_state(w, N=n)
    p, op = _pair(imrp, w, n, precision=prec, nu_coll=2.0)
    assert op.nu_coll == 2.0
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        q, u = sim.step(5)
        xg, vg = sim.particles()
    xo, vo, qo, uo, hits = oracle.run(op, x, v, 5)
    # velocity after the collisions of the last step: a scattered particle's
    # direction is new, so a different decision would show as an O(1) change
    dv_g, dv_o = vg - v, vo - v
    per = np.linalg.norm(dv_g - dv_o, axis=1) / (np.linalg.norm(vo, axis=1) + 1e-30)
    bad = np.sum(per > 1e-2)
    assert bad <= (0 if prec == 0 else 2), f"{bad} particles differ"
    good = per <= 1e-2
    assert _rel(vg[good], vo[good]) < TOL[prec] * 10
    assert _rel(xg[good], xo[good]) < TOL[prec]
    # speeds change only through the field and the walls: scattering keeps them
    scattered = np.sum(np.abs(np.einsum("ij,ij->i", vo, v) / (np.linalg.norm(vo, axis=1) * np.linalg.norm(v, axis=1))) < 0.9)
    assert scattered > 0.2 * n


@pytest.mark.parametrize("prec", [0, 1])
def test_absorbing_walls_match_oracle(imrp, prec):
    """wall_rule = 2: electrons that reach the probe are absorbed and their
    charge joins Q_S, those that reach the outer wall leave, and each is
    replaced from the outer wall with the same Philox draws on both sides.
    Six steps: positions, velocities, Q_diff, the surface charge and the
    absorption count against the oracle's run."""
    n = 3000
    # a narrow shell (1 < r < 1.6) of hot electrons, so that many reach each wall
    w = Workload("absorb", N=n, l_max=8, T_e_eV=20.0, n_e_m3=1e15, outer_R=1.6, drive_kind=1,
                 V_volts=50.0, wall_rule=2)
    x, v = workload_state(w, N=n)
    p, op = _pair(imrp, w, n, precision=prec)
    assert op.wall_rule == 2 and op.sigma_v > 0
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        q, u = sim.step(6)
        xg, vg = sim.particles()
        qs_g, nab_g = sim.surface_charge()
    xo, vo, qo, uo, hits, qs_o, nab_o = oracle.run(op, x, v, 6, surface=True)
    assert nab_o > 5 and hits > nab_o
    # the same particles are absorbed (an FP32 radius within rounding of a wall
    # may decide otherwise on the mixed path)
    assert abs(nab_g - nab_o) <= (0 if prec == 0 else 2)
    assert qs_g == -nab_g and qs_o == -nab_o
    per = np.linalg.norm(xg - xo, axis=1) / np.linalg.norm(xo, axis=1)
    bad = np.sum(per > 10 * TOL[prec])
    assert bad <= (0 if prec == 0 else 3), f"{bad} particles differ"
    good = per <= 10 * TOL[prec]
    assert _rel(xg[good], xo[good]) < TOL[prec]
    assert _rel(vg[good], vo[good]) < 10 * TOL[prec]
    np.testing.assert_allclose(q, qo, rtol=10 * TOL[prec], atol=10 * TOL[prec] * np.max(np.abs(qo)))
    # every particle is inside the domain, and the re-injected ones moved inwards
    r = np.linalg.norm(xg, axis=1)
    assert np.all((r >= 1.0) & (r <= op.r_out * (1 + 1e-6)))


def test_qdiff_and_drive_sequence(imrp):
    """FP64 path: 40 steps of the Gaussian pulse stay on the oracle trajectory."""
    n = 1200
    x, v = workload_state(BASE, N=n)
    p, op = _pair(imrp, BASE, n, precision=0, l_max=4)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        q1, u1 = sim.step(17)   # odd: graph pairs and a one-step graph
        q2, u2 = sim.step(23)
        qa, ua = sim.qdiff()
    xo, vo, qo, uo, _ = oracle.run(op, x, v, 40)
    np.testing.assert_allclose(np.concatenate([u1, u2]), uo, rtol=1e-12)
    np.testing.assert_allclose(qa, np.concatenate([q1, q2]), rtol=0, atol=0)
    np.testing.assert_allclose(qa, qo, rtol=1e-6, atol=1e-9 * np.max(np.abs(qo)))


@pytest.mark.parametrize("prec", [0, 1])
def test_single_steps_pairs_and_reloads_agree(imrp, prec):
    """Captured one-step and two-step graphs replay the same kernels: five
    single steps, one call of five steps, and a context that first ran another
    state of the same size and then reloaded (keeping its captured graphs)
    give bitwise the same particles and Q_diff."""
    n = 3001
    x, v = workload_state(BASE, N=n)
    x2, v2 = workload_state(BASE, N=n)[0][::-1].copy(), workload_state(BASE, N=n)[1][::-1].copy()
    p, _ = _pair(imrp, BASE, n, precision=prec, l_max=8)
    with imrp.Sim(p) as a, imrp.Sim(p) as b, imrp.Sim(p) as c:
        a.load(x, v)
        for _ in range(5):
            a.step(1)
        b.load(x, v)
        b.step(5)
        c.load(x2, v2)
        c.step(3)
        c.load(x, v)
        c.step(5)
        xa, va = a.particles()
        xb, vb = b.particles()
        xc, vc = c.particles()
        qa, qb, qc = a.qdiff()[0], b.qdiff()[0], c.qdiff()[0]
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(xc, xb)
    np.testing.assert_array_equal(vc, vb)
    np.testing.assert_array_equal(qa, qb)
    np.testing.assert_array_equal(qc, qb)


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_restore_continues_bitwise(imrp, prec):
    """A run checkpointed after 7 steps and restored into a fresh context
    continues bit for bit: diffuse walls and collisions draw from counters of
    (seed, id, step), the Gaussian pulse is a function of the step, and the
    storage order keeps the order of equal keys."""
    n = 3001
    w = Workload("walls", N=n, l_max=8, T_e_eV=20.0, n_e_m3=1e15, drive_kind=0, V_volts=50.0)
    x, v = workload_state(w, N=n)
    p, _ = _pair(imrp, w, n, precision=prec, nu_coll=0.5)
    with imrp.Sim(p) as a, imrp.Sim(p) as b:
        a.load(x, v)
        a.step(7)
        ck = a.checkpoint()
        assert ck[3] == 7 and sorted(ck[2].tolist()) == list(range(n))
        a.step(6)
        xa, va = a.particles()
        qa, ua = a.qdiff(7, 6)
        b.restore(*ck)
        b.step(5)
        b.step(1)
        xb, vb = b.particles()
        qb, ub = b.qdiff(7, 6)
        with pytest.raises(imrp.IMRPError):
            b.qdiff(0, 3)        # before the restored step: not recorded here
        with pytest.raises(imrp.IMRPError):
            b.spectrum()         # needs the series from the drive
        bad = ck[2].copy()
        bad[0] = bad[1]
        with pytest.raises(imrp.IMRPError):
            b.restore(ck[0], ck[1], bad, ck[3])
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(qa, qb)
    np.testing.assert_array_equal(ua, ub)


def test_errors_are_reported(imrp):
    p = imrp.params_from_workload(BASE, N=100)
    with imrp.Sim(p) as sim:
        with pytest.raises(imrp.IMRPError) as e:
            sim.step(1)
        assert e.value.code == -6
        x, v = workload_state(BASE, N=100)
        x[5] *= 0.5  # inside the probe
        with pytest.raises(imrp.IMRPError) as e:
            sim.load(x, v)
        assert e.value.code == -1
        with pytest.raises(imrp.IMRPError):
            sim.load(np.zeros((200, 3)), np.zeros((200, 3)))
    bad = imrp.params_from_workload(BASE, N=100, l_max=7)
    with pytest.raises(imrp.IMRPError):
        imrp.Sim(bad)


def test_large_sampled_parity(imrp):
    """The mixed-precision workload at full size (N = 2e6, l_max = 16): sampled
    particles against the oracle's direct pair sum, and invariants after a step."""
    w = WORKLOADS["mixed_n2e6_l16"]
    x, v = workload_state(w)
    p, op = _pair(imrp, w, w.N)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        E = sim.field()
        q, _ = sim.step(2)
        xg, vg = sim.particles()
    rng = np.random.default_rng(0)
    # spread the samples over the radius order (inner, middle and outer tiles)
    order = np.argsort(np.linalg.norm(x, axis=1))
    sample = np.unique(np.concatenate([order[:3], order[-3:], rng.choice(w.N, 10, replace=False)]))
    Eo = oracle.field_brute(op, x, u=oracle.drive(op, 0), sample=sample)
    rel = _rel(E[sample], Eo)
    err = np.linalg.norm(E[sample] - Eo, axis=1) / np.linalg.norm(Eo, axis=1)
    print(f"N=2e6 sampled: ||dE||/||E|| = {rel:.3e}, largest per particle {err.max():.3e}")
    assert rel < TOL[1]
    assert err.max() < P999[1]
    r = np.linalg.norm(xg, axis=1)
    assert np.all(r >= 1.0) and np.all(r <= op.r_out)
    assert np.all(np.isfinite(vg)) and np.all(np.isfinite(q))


@pytest.mark.parametrize("prec", [0, 1])
def test_field_on_reused_device_memory(imrp, prec):
    """A context created where an earlier one's buffers were freed (the device
    allocator hands the same memory back, so the tile-sum arrays start with
    the earlier instance's values): every tile the scans read must be written,
    including the empty tiles of a ragged last scan group (n = 2500 fills 79
    of the group's 96 tiles)."""
    big = WORKLOADS["fp64_n2e4_l8"]
    for n_prev in (20000, 9001):
        x0, v0 = workload_state(big, N=n_prev)
        with imrp.Sim(imrp.params_from_workload(big, N=n_prev, precision=prec)) as s0:
            s0.load(x0, v0)
            s0.step(2)
        n = 2500
        x, v = workload_state(big, N=n)
        p, op = _pair(imrp, big, n, precision=prec)
        with imrp.Sim(p) as sim:
            sim.load(x, v)
            E = sim.field()
        Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
        check_field(E, Eo, prec, f"reused memory after n={n_prev}")


def test_fp32_load_rounds_to_nearest_even(imrp):
    """The load converts FP64 host data to the FP32 state by round to nearest,
    ties to even (its own integer rounding in the normal range, the hardware
    conversion elsewhere): bit for bit what numpy's float32 conversion gives,
    on exact ties both ways, carries into the exponent, values near the top of
    the FP32 range and past it (infinity), subnormal results and the ties
    between them and zero, signed zeros."""
    rng = np.random.default_rng(4)
    n = 4096
    w = WORKLOADS["fp64_n2e4_l8"]
    x, v = workload_state(w, N=n)
    x = x.copy()
    v = v.copy()
    # ties: a float32 value plus or minus half its spacing (even and odd mantissas)
    f = x[:1024].astype(np.float32)
    half = np.spacing(f).astype(np.float64) / 2
    x[:512] = f[:512].astype(np.float64) + half[:512]
    x[512:1024] = f[512:1024].astype(np.float64) - half[512:1024]
    # velocities: random bits of the mantissa, carries, extremes
    vv = v.reshape(-1)
    vv[:3000] = rng.standard_normal(3000) * np.exp(rng.uniform(-20, 20, 3000))
    edge = np.array([np.nextafter(2.0, 0.0), np.nextafter(1.0, 2.0), -np.nextafter(4.0, 0.0), 3.3e38,
                     -3.4e38, float(np.float32(3.4028235e38)) * (1 - 2 ** -25), 1e-40, -3e-45, 1e-46,
                     0.0, -0.0, 1.1754942e-38, 1.1754944e-38, 5.877472e-39, 3.5e38, -1e39,
                     1.401298464324817e-45 * 0.5, 1.401298464324817e-45 * 0.75, 1.401298464324817e-45 * 1.5])
    vv[3000:3000 + edge.size] = edge
    p = imrp.params_from_workload(w, N=n, precision=1)
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        xg, vg = sim.particles()
    with np.errstate(over="ignore"):
        xf, vf = x.astype(np.float32), v.astype(np.float32)
    np.testing.assert_array_equal(xg, xf.astype(np.float64))
    np.testing.assert_array_equal(vg, vf.astype(np.float64))
    assert np.array_equal(np.signbit(vg), np.signbit(vf))


def test_large_sampled_parity_fp64(imrp):
    """FP64 at N = 2e6, l_max = 8: the moments kernel's 1024-particle blocks
    (an FP64 instance this large fills the GPU with them; smaller FP64
    instances use 256-particle blocks, covered by the full comparisons above),
    sampled particles against the oracle's direct pair sum."""
    w = WORKLOADS["mixed_n2e6_l16"]
    x, _ = workload_state(w)
    p, op = _pair(imrp, w, w.N, precision=0, l_max=8)
    with imrp.Sim(p) as sim:
        sim.load(x, np.zeros_like(x))
        E = sim.field()
    rng = np.random.default_rng(1)
    order = np.argsort(np.linalg.norm(x, axis=1))
    sample = np.unique(np.concatenate([order[:2], order[-2:], rng.choice(w.N, 8, replace=False)]))
    Eo = oracle.field_brute(op, x, u=oracle.drive(op, 0), sample=sample)
    err = np.linalg.norm(E[sample] - Eo, axis=1) / np.linalg.norm(Eo, axis=1)
    print(f"N=2e6 FP64 sampled: largest per particle {err.max():.3e}")
    assert _rel(E[sample], Eo) < TOL[0]
    assert err.max() < P999[0]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L,si,drive", [(1, 0, 1), (1, 1, 1), (4, 0, 2), (8, 1, 1), (16, 0, 1)])
def test_m0_only_truncation_matches_oracle(imrp, prec, L, si, drive):
    """The paper's truncation (Sec. 3: m = 0 terms only; with l_max = 1 the printed
    cos t cos t' kernel), self image on and off, with a strong impulse drive."""
    n = 3001
    x, v = workload_state(BASE, N=n)
    p, op = _pair(imrp, BASE, n, precision=prec, l_max=L, m0_only=1, self_image=si,
                  drive_kind=drive, V_volts=200.0)
    op.m0_only = 1
    with imrp.Sim(p) as sim:
        sim.load(x, v)
        E = sim.field()
        q, _ = sim.step(3)
        xg, vg = sim.particles()
    Eo = oracle.field_scan(op, x, u=oracle.drive(op, 0))
    check_field(E, Eo, prec, f"m0_only L={L}")
    xo, vo, qo, _, _ = oracle.run(op, x, v, 3)
    assert _rel(vg - v, vo - v) < 10 * TOL[prec]
    np.testing.assert_allclose(q, qo, rtol=10 * TOL[prec], atol=10 * TOL[prec] * np.max(np.abs(qo)))

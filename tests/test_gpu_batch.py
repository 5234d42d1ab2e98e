"""Batched ensembles and the autotuner.

A context stepped inside a batch (one captured graph across contexts of uneven
N, degree and precision, with the moments and the field of all contexts of a
degree and precision in one launch over a work list of (context, block))
computes exactly what it computes alone: Q_diff and the final state are
bit-identical. Autotuning changes only launch shapes, never the
arithmetic of a particle: the field is bit-identical before and after.
"""
import numpy as np
import pytest

from paper_2111_13072_gb300.inputs import Workload, workload_state

pytestmark = pytest.mark.gpu

CASES = [  # (N, l_max, T_e, n_e, precision, seed); several share a degree and precision,
    # so that their moments and field run in one batched launch
    (1000, 4, 2.0, 1e15, 0, 1),
    (33000, 8, 0.5, 3e14, 1, 2),
    (12345, 12, 5.0, 1e17, 1, 3),
    (70000, 16, 3.0, 1e16, 1, 4),
    (5000, 8, 2.0, 1e15, 0, 5),
    (9001, 8, 1.0, 1e15, 1, 6),
    (2047, 16, 4.0, 1e16, 1, 7),
    (700, 16, 2.0, 1e15, 1, 8),
]


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    return m


def _make(imrp, case, wall_rule=0, ions=False):
    N, L, T, n, prec, seed = case
    w = Workload("b", N=N, l_max=L, T_e_eV=T, n_e_m3=n, precision=prec, seed=seed, wall_rule=wall_rule)
    x, v = workload_state(w)
    s = imrp.Sim(imrp.params_from_workload(w))
    if ions:
        s.set_species(N - N // 3, 1.0, 50.0, float(N - 2 * (N // 3)))
    s.load(x, v)
    return s


@pytest.mark.parametrize("nsteps", [21, 4])
def test_batch_equals_alone(imrp, nsteps):
    alone = []
    for c in CASES:
        with _make(imrp, c) as s:
            q, u = s.step(nsteps)
            x, v = s.particles()
            alone.append((q, x, v))
    sims = [_make(imrp, c) for c in CASES]
    with imrp.Batch(sims) as b:
        b.step(nsteps // 2)
        b.step(nsteps - nsteps // 2)
        b.sync()
    for s, (q0, x0, v0) in zip(sims, alone):
        q, _ = s.qdiff()
        x, v = s.particles()
        np.testing.assert_array_equal(q, q0)
        np.testing.assert_array_equal(x, x0)
        np.testing.assert_array_equal(v, v0)
        s.close()


def test_batch_with_absorbing_walls_and_ions_equals_alone(imrp):
    """Contexts with the absorbing wall (Q_S accrues from the batched field
    launch's absorptions) and with mobile ions (charge scans per context
    between the batched launches), batched with a plain one of the same degree."""
    specs = [(dict(case=(6000, 8, 20.0, 1e15, 1, 11), wall_rule=2)),
             (dict(case=(4001, 8, 3.0, 1e15, 1, 12), ions=True)),
             (dict(case=(3000, 8, 2.0, 1e15, 1, 13)))]
    alone = []
    for sp in specs:
        with _make(imrp, **sp) as s:
            q, _ = s.step(6)
            alone.append((q, s.particles()[0], s.surface_charge()))
    sims = [_make(imrp, **sp) for sp in specs]
    with imrp.Batch(sims) as b:
        b.step(6)
        b.sync()
    for s, (q0, x0, qs0) in zip(sims, alone):
        np.testing.assert_array_equal(s.qdiff()[0], q0)
        np.testing.assert_array_equal(s.particles()[0], x0)
        assert s.surface_charge() == qs0
        s.close()
    assert alone[0][2][1] > 0  # the absorbing wall took electrons in the hot shell


def test_autotune_keeps_results(imrp):
    s = _make(imrp, CASES[3])
    E0 = s.field()
    w, c = s.autotune()
    assert w in (1, 2, 4, 8) and c in (16, 32, 64)
    E1 = s.field()
    np.testing.assert_array_equal(E0, E1)
    q, _ = s.step(6)
    assert np.all(np.isfinite(q))
    s.close()


def test_autotune_is_not_slower(imrp):
    """The autotuner times the field kernel at every CTA size, the default
    among them, and keeps the fastest: the field stage after tuning is no
    slower than before (medians of three timed runs of 20 steps each, N = 2e5
    at l_max = 16, 10 % allowed for run-to-run noise)."""
    s = _make(imrp, (200000, 16, 3.0, 1e16, 1, 9))

    def field_ms():
        return float(np.median([s.profile_steps(20)["field"] for _ in range(3)]))

    s.profile_steps(5)  # warm-up
    before = field_ms()
    s.autotune()
    after = field_ms()
    print(f"field stage: {before:.4f} ms before tuning, {after:.4f} ms after")
    assert after <= 1.10 * before
    s.close()


def test_batch_autotune_keeps_results(imrp):
    """The batch autotuner picks a CTA size per batched field launch; steps
    after it are bit-identical to steps of the same contexts alone, and a
    batch captured before tuning is recaptured with the tuned shapes."""
    cases = CASES[1:6]
    alone = []
    for c in cases:
        with _make(imrp, c) as s:
            q, _ = s.step(6)
            alone.append((q, s.particles()[0]))
    sims = [_make(imrp, c) for c in cases]
    with imrp.Batch(sims) as b:
        b.step(2)
        b.autotune()
        b.step(3)
        b.autotune()
        b.step(1)
        b.sync()
    for s, (q0, x0) in zip(sims, alone):
        np.testing.assert_array_equal(s.qdiff()[0], q0)
        np.testing.assert_array_equal(s.particles()[0], x0)
        s.close()

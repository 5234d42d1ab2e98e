"""Batched ensembles and the autotuner.

A context stepped inside a batch (one captured graph across contexts of uneven
N, degree and precision) computes exactly what it computes alone: Q_diff and the
final state are bit-identical. Autotuning changes only launch shapes, never the
arithmetic of a particle: the field is bit-identical before and after.
"""
import numpy as np
import pytest

from paper_2111_13072_gb300.inputs import Workload, workload_state

pytestmark = pytest.mark.gpu

CASES = [  # (N, l_max, T_e, n_e, precision, seed)
    (1000, 4, 2.0, 1e15, 0, 1),
    (33000, 8, 0.5, 3e14, 1, 2),
    (12345, 12, 5.0, 1e17, 1, 3),
    (70000, 16, 3.0, 1e16, 1, 4),
    (5000, 8, 2.0, 1e15, 0, 5),
]


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    return m


def _make(imrp, case):
    N, L, T, n, prec, seed = case
    w = Workload("b", N=N, l_max=L, T_e_eV=T, n_e_m3=n, precision=prec, seed=seed)
    x, v = workload_state(w)
    s = imrp.Sim(imrp.params_from_workload(w))
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


def test_autotune_keeps_results(imrp):
    s = _make(imrp, CASES[3])
    E0 = s.field()
    w, c = s.autotune()
    assert w in (1, 2, 4, 8) and c in (8, 16, 32)
    E1 = s.field()
    np.testing.assert_array_equal(E0, E1)
    q, _ = s.step(6)
    assert np.all(np.isfinite(q))
    s.close()

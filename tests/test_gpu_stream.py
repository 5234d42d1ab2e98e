"""Streamed loads (imrp_load_particles_async) and queued Q_diff read-back
(imrp_copy_qdiff_async): the same results as the synchronous calls, bit for
bit, with the copies of the next particle set overlapping the steps in flight,
and range errors reported by the next synchronising call."""
import numpy as np
import pytest

from paper_2111_13072_gb300.inputs import WORKLOADS, Workload, workload_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available(), "these tests need the GPU"
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


@pytest.mark.parametrize("prec", [0, 1])
def test_streamed_loads_match_synchronous(imrp, prec):
    import torch
    w = WORKLOADS["fp64_n2e4_l8"]
    n, k = 5000, 4
    sets = [workload_state(Workload("s", N=n, l_max=8, T_e_eV=2.0, n_e_m3=1e15, seed=s), N=n) for s in range(k)]
    p = imrp.params_from_workload(w, N=n, precision=prec, drive_kind=1, V_volts=30.0)
    # synchronous reference: load, 3 steps, Q_diff, for each set
    ref = []
    with imrp.Sim(p) as sim:
        for x, v in sets:
            sim.load(x, v)
            q, _ = sim.step(3)
            ref.append(q)
    # streamed: every load and step queued before any result is read
    xs = [torch.from_numpy(x).pin_memory() for x, _ in sets]
    vs = [torch.from_numpy(v).pin_memory() for _, v in sets]
    qh = torch.zeros(k, 3, dtype=torch.float64).pin_memory()
    with imrp.Sim(p) as sim:
        for i in range(k):
            sim.load_async_ptr(xs[i].data_ptr(), vs[i].data_ptr(), n)
            sim.step_async(3)
            sim.copy_qdiff_async(0, 3, qh[i].data_ptr())
        sim.sync()
    np.testing.assert_array_equal(qh.numpy(), np.array(ref))


def test_streamed_load_reports_bad_particles(imrp):
    import torch
    w = WORKLOADS["fp64_n2e4_l8"]
    n = 1000
    x, v = workload_state(w, N=n)
    x[7] *= 0.5 / np.linalg.norm(x[7])  # r = 0.5: inside the probe
    p = imrp.params_from_workload(w, N=n)
    xt, vt = torch.from_numpy(x).pin_memory(), torch.from_numpy(v).pin_memory()
    with imrp.Sim(p) as sim:
        sim.load_async_ptr(xt.data_ptr(), vt.data_ptr(), n)
        with pytest.raises(imrp.IMRPError) as e:
            sim.sync()
        assert e.value.code == -1
        with pytest.raises(imrp.IMRPError) as e:
            sim.load_async_ptr(xt.data_ptr(), vt.data_ptr(), 10 * n)
        assert e.value.code == -1

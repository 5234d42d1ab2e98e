"""Seeded synthetic inputs: shape of the workload (Sec. 4 units)."""
import numpy as np

from paper_2111_13072_gb300.inputs import WORKLOADS, debye_length_m, maxwellian_shell, workload_state


def test_shell_positions_and_velocities():
    x, v = maxwellian_shell(50000, 2.3, 0.05, seed=3)
    r = np.linalg.norm(x, axis=1)
    assert r.min() > 1.0 and r.max() < 2.3
    # uniform in volume: the fraction inside the mid-volume radius is ~1/2
    rm = ((1 + 2.3 ** 3) / 2) ** (1 / 3)
    assert abs(np.mean(r < rm) - 0.5) < 0.01
    assert abs(np.std(v) - 0.05) < 0.001
    np.testing.assert_array_equal(x, x.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(v, v.astype(np.float32).astype(np.float64))


def test_seeded_and_prefix_free_of_state():
    a = maxwellian_shell(1000, 2.0, 0.1, seed=7)
    b = maxwellian_shell(1000, 2.0, 0.1, seed=7)
    c = maxwellian_shell(1000, 2.0, 0.1, seed=8)
    np.testing.assert_array_equal(a[0], b[0])
    assert not np.array_equal(a[0], c[0])


def test_workload_geometry():
    w = WORKLOADS["fp64_n2e4_l8"]
    lam = debye_length_m(1e15, 2.0)
    assert abs(lam - 3.3245e-4) < 1e-7
    assert abs(w.r_out - (5e-3 + 20 * lam) / 5e-3) < 1e-12
    x, v = workload_state(w, N=100)
    assert x.shape == (100, 3)

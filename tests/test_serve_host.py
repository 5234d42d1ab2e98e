"""Host-side request and ensemble generators (no GPU)."""
import numpy as np

from paper_2111_13072_gb300.serve import ensemble_workloads, serving_requests


def test_serving_requests_distribution():
    rs = serving_requests(400, rate=20.0, steps=100, seed=5)
    t = np.array([r.arrival for r in rs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(rs) / t[-1] - 20.0) < 3.0
    N = np.array([r.workload.N for r in rs])
    assert N.min() >= 1e5 and N.max() <= 4e6
    assert {r.workload.l_max for r in rs} == {8, 16}
    assert all(0.5 <= r.workload.T_e_eV <= 5.0 for r in rs)
    assert all(1e14 <= r.workload.n_e_m3 <= 1e17 for r in rs)
    rs2 = serving_requests(400, rate=20.0, steps=100, seed=5)
    assert [r.workload.N for r in rs2] == list(N)


def test_ensemble_workloads():
    ws = ensemble_workloads(64, seed=3)
    assert len(ws) == 64
    N = np.array([w.N for w in ws])
    assert N.min() >= 1e4 and N.max() <= 1e6
    assert {w.l_max for w in ws} <= {8, 12, 16}

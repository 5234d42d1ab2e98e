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


class _FakeError(RuntimeError):
    pass


class _FakeSim:
    """Stands in for a GPU context: counts steps, fails (a device error flag
    that the batch check reports) once it passes fail_at."""

    def __init__(self, params):
        self.n_steps = params["steps"]
        self.fail_at = params["fail_at"]
        self.step = 0
        self.flag = False
        self.closed = False

    def load(self, x, v):
        pass

    def sync(self):
        if self.flag:
            self.flag = False
            raise _FakeError("IMRP_E_NAN: non-finite value in the particle state")

    def spectrum(self, n_freq, w_max):
        return {"w_res": 0.5, "dw": 0.1, "fit": np.zeros(4), "omega": np.zeros(3), "reY": np.zeros(3)}

    def qdiff(self):
        return np.zeros(self.step), np.zeros(self.step)

    def close(self):
        self.closed = True


class _FakeBatch:
    def __init__(self, sims):
        self.sims = sims
        self.failed = -1

    def step(self, n):
        for s in self.sims:
            assert not s.closed
            s.step += n
            if s.fail_at is not None and s.step > s.fail_at:
                s.flag = True

    def sync(self):
        self.failed = -1
        for i, s in enumerate(self.sims):
            if s.flag:
                s.flag = False  # the report clears the first failing context's flags
                self.failed = i
                raise _FakeError("IMRP_E_NAN: non-finite value in the particle state")

    def failed_index(self):
        return self.failed

    def close(self):
        pass


class _FakeBackend:
    IMRPError = _FakeError
    Sim = _FakeSim
    Batch = _FakeBatch

    def __init__(self, fail):
        self.fail = fail
        self.sims = {}

    def params_from_workload(self, w):
        return {"steps": w.steps, "fail_at": self.fail.get(w.name)}

    def footprint(self, params, steps):
        return 1000


def test_server_evicts_failing_requests_and_serves_the_rest():
    """Failure detection on the host: two of five requests' contexts report a
    device error mid-run (both in the same chunk); they are evicted with the
    error, their memory returns, and the other three finish their steps."""
    from paper_2111_13072_gb300.inputs import Workload
    from paper_2111_13072_gb300.serve import SpectrumRequest, SpectrumServer

    fail = {"r1": 250, "r3": 260}
    reqs = [SpectrumRequest(i, Workload(f"r{i}", N=10, l_max=1, T_e_eV=1.0, n_e_m3=1e15, steps=1000),
                            steps=1000, arrival=0.0) for i in range(5)]
    backend = _FakeBackend(fail)
    srv = SpectrumServer(hbm_budget=10 ** 6, chunk=100, backend=backend,
                         state_fn=lambda w: (np.zeros((w.N, 3)), np.zeros((w.N, 3))))
    res = srv.serve(reqs, realtime=False)
    assert [r.rid for r in res] == [0, 1, 2, 3, 4]
    errs = {r.rid: r.error for r in res}
    assert errs[1] and "IMRP_E_NAN" in errs[1]
    assert errs[3] and "IMRP_E_NAN" in errs[3]
    assert errs[0] is None and errs[2] is None and errs[4] is None
    assert srv.stats["evicted"] == 2
    for r in res:
        if r.error is None:
            assert len(r.qdiff) == 1000  # every step done, none twice
            assert r.w_res == 0.5


def test_server_reraises_errors_of_the_batch_itself():
    from paper_2111_13072_gb300.inputs import Workload
    from paper_2111_13072_gb300.serve import SpectrumRequest, SpectrumServer

    class Broken(_FakeBatch):
        def sync(self):
            self.failed = -1
            raise _FakeError("IMRP_E_CUDA: sync")

    backend = _FakeBackend({})
    backend.Batch = Broken
    srv = SpectrumServer(hbm_budget=10 ** 6, chunk=100, backend=backend,
                         state_fn=lambda w: (np.zeros((w.N, 3)), np.zeros((w.N, 3))))
    req = SpectrumRequest(0, Workload("r0", N=10, l_max=1, T_e_eV=1.0, n_e_m3=1e15, steps=200), steps=200)
    try:
        srv.serve([req], realtime=False)
    except _FakeError as e:
        assert "sync" in str(e)
    else:
        raise AssertionError("a batch error must propagate")

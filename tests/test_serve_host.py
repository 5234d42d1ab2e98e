"""Host side of the serving and ensemble workloads (no GPU): the request and
ensemble generators, and the serving loop driven by a fake backend (failure
detection, independent progress, memory admission, error propagation)."""
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
    that its sync reports) once it passes fail_at; its queued chunk is done
    after `delay` polls."""

    def __init__(self, params):
        self.n_steps = params["steps"]
        self.fail_at = params["fail_at"]
        self.broken = params["broken"]
        self.step = 0
        self.flag = False
        self.closed = False
        self.busy = 0
        self.delay = params["delay"]

    def load(self, x, v):
        pass

    def step_async(self, n):
        assert not self.closed
        if self.broken:
            raise _FakeError("IMRP_E_CUDA: launch")
        self.step += n
        self.busy = self.delay
        if self.fail_at is not None and self.step > self.fail_at:
            self.flag = True

    def ready(self):
        if self.busy:
            self.busy -= 1
            return False
        return True

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


class _FakeBackend:
    IMRPError = _FakeError
    Sim = _FakeSim

    def __init__(self, fail, broken=(), delays=None):
        self.fail = fail
        self.broken = set(broken)
        self.delays = delays or {}

    def params_from_workload(self, w):
        return {"steps": w.steps, "fail_at": self.fail.get(w.name), "broken": w.name in self.broken,
                "delay": self.delays.get(w.name, 1)}

    def footprint(self, params, steps):
        return 1000


def _server(backend, **kw):
    from paper_2111_13072_gb300.serve import SpectrumServer
    return SpectrumServer(hbm_budget=kw.pop("budget", 10 ** 6), chunk=100, backend=backend, poll_s=0.0,
                          state_fn=lambda w: (np.zeros((w.N, 3)), np.zeros((w.N, 3))), **kw)


def _reqs(n, steps=1000):
    from paper_2111_13072_gb300.inputs import Workload
    from paper_2111_13072_gb300.serve import SpectrumRequest
    return [SpectrumRequest(i, Workload(f"r{i}", N=10, l_max=1, T_e_eV=1.0, n_e_m3=1e15, steps=steps),
                            steps=steps, arrival=0.0) for i in range(n)]


def test_server_evicts_failing_requests_and_serves_the_rest():
    """Failure detection on the host: two of five requests' contexts report a
    device error mid-run (in the same chunk); they are evicted with the error,
    their memory returns, and the other three finish their steps."""
    backend = _FakeBackend({"r1": 250, "r3": 260})
    srv = _server(backend)
    res = srv.serve(_reqs(5), realtime=False)
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


def test_requests_progress_independently():
    """A slow request (its chunks take many polls) does not hold back a fast
    one: the fast request finishes first although both were admitted together,
    and both run every step exactly once."""
    backend = _FakeBackend({}, delays={"r0": 50, "r1": 0})
    res = _server(backend).serve(_reqs(2), realtime=False)
    assert res[1].finished < res[0].finished
    assert [len(r.qdiff) for r in res] == [1000, 1000]


def test_admission_waits_for_memory():
    """With room for two requests at a time, the third is admitted only once
    one of the first two has finished and returned its memory."""
    backend = _FakeBackend({})
    srv = _server(backend, budget=2000)
    res = srv.serve(_reqs(3, steps=300), realtime=False)
    assert srv.stats["peak_bytes"] <= 2000
    assert srv.stats["max_active"] == 2
    assert res[2].admitted >= min(res[0].finished, res[1].finished)


def test_server_reraises_errors_that_are_not_one_requests():
    backend = _FakeBackend({}, broken={"r0"})
    srv = _server(backend)
    try:
        srv.serve(_reqs(1, steps=200), realtime=False)
    except _FakeError as e:
        assert "launch" in str(e)
    else:
        raise AssertionError("a launch error must propagate")

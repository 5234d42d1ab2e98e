"""Continuous-batching spectrum service: requests admitted while others run
return exactly what they return alone, and admission respects the memory
budget."""
import numpy as np
import pytest

from paper_2111_13072_gb300.inputs import Workload, workload_state

pytestmark = pytest.mark.gpu


def _requests(serve):
    specs = [(3000, 4, 2.0, 1e15, 40, 0.0), (20000, 8, 0.5, 3e14, 60, 0.0),
             (7000, 8, 4.0, 1e16, 50, 1e-9), (11000, 4, 1.0, 1e17, 30, 2e-9)]
    out = []
    for i, (N, L, T, n, steps, t) in enumerate(specs):
        w = Workload(f"r{i}", N=N, l_max=L, T_e_eV=T, n_e_m3=n, precision=i % 2, seed=100 + i)
        out.append(serve.SpectrumRequest(i, w, steps, arrival=t, n_freq=300, w_max=1.5))
    return out


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp, serve
    build.build()
    return imrp, serve


def test_results_in_the_mix_equal_alone(mods):
    imrp, serve = mods
    reqs = _requests(serve)
    srv = serve.SpectrumServer(chunk=10)
    res = srv.serve(reqs, realtime=False)
    assert len(res) == len(reqs)
    assert srv.stats["max_active"] >= 3  # late arrivals joined running requests
    for r, req in zip(res, reqs):
        with imrp.Sim(imrp.params_from_workload(req.workload)) as s:
            x, v = workload_state(req.workload)
            s.load(x, v)
            q, _ = s.step(req.steps)
            sp = s.spectrum(req.n_freq, req.w_max)
        np.testing.assert_array_equal(r.qdiff, q)
        np.testing.assert_array_equal(r.reY, sp["reY"])
        assert r.w_res == sp["w_res"] and r.dw == sp["dw"]


def test_admission_respects_memory_budget(mods):
    imrp, serve = mods
    reqs = _requests(serve)
    fps = [imrp.footprint(imrp.params_from_workload(r.workload), r.steps) for r in reqs]
    budget = sorted(fps)[-1] + sorted(fps)[-2]  # room for the two largest at once
    srv = serve.SpectrumServer(hbm_budget=budget, chunk=10)
    res = srv.serve(reqs, realtime=False)
    assert len(res) == len(reqs)
    assert srv.stats["peak_bytes"] <= budget
    assert all(r.finished >= r.admitted >= r.arrival for r in res)

"""imrp_field_noalloc: the field evaluation for callers that cannot allocate
device memory (a framework that owns every device buffer through its own pool,
a service loop that must not grow device memory after start-up). Called
through the C ABI on caller-owned device buffers, twice in a row with
different particle sets, it must return what the allocating path
(imrp_get_field on a context) returns, within the parity tolerance of the
precision. This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2111_13072_gb300.inputs import WORKLOADS, workload_state

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-4}


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_context_field_twice(prec):
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp
    build.build()
    w = WORKLOADS["fp64_n2e4_l8"]
    stream = torch.cuda.Stream()
    for n, L, seed in ((9001, 8, 11), (3001, 16, 12)):  # second call: smaller n, other degree
        x, v = workload_state(w, N=n)
        x = x[np.random.default_rng(seed).permutation(n)]
        p = imrp.params_from_workload(w, N=n, precision=prec, l_max=L, drive_kind=1, V_volts=40.0)
        with imrp.Sim(p) as sim:
            sim.load(x, v)
            E_ref = sim.field()
        xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
        Ed = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        imrp.field_noalloc(p, xd.data_ptr(), n, 0, Ed.data_ptr(), stream.cuda_stream)
        E = Ed.cpu().numpy()
        rel = np.linalg.norm(E - E_ref) / np.linalg.norm(E_ref)
        assert rel < TOL[prec], (n, L, rel)


def test_noalloc_rejects_beyond_limits():
    import torch
    from paper_2111_13072_gb300 import imrp
    w = WORKLOADS["fp64_n2e4_l8"]
    p = imrp.params_from_workload(w, N=10)
    xd = torch.ones(20000, 3, dtype=torch.float64, device="cuda") * 1.2
    Ed = torch.empty(20000, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(imrp.IMRPError) as e:
        imrp.field_noalloc(p, xd.data_ptr(), 20000, 0, Ed.data_ptr())
    assert e.value.code == -1
    p24 = imrp.params_from_workload(w, N=10, l_max=24)
    with pytest.raises(imrp.IMRPError):
        imrp.field_noalloc(p24, xd.data_ptr(), 100, 0, Ed.data_ptr())

"""imrp_field_noalloc: the field evaluation for callers that cannot allocate
device memory (a framework that owns every device buffer through its own pool,
a service loop that must not grow device memory after start-up). Called
through the C ABI on caller-owned device buffers, several times in a row with
different particle sets, degrees and steps, it must return what the allocating
path (imrp_get_field on a context) returns and what the FP64 oracle returns,
within the parity tolerance of the precision; and after its first call on the
device (the set-up, which loads the device code and reserves the static
scratch) it must not change the device's free memory or the caching
allocator's statistics. This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2111_13072_gb300.inputs import WORKLOADS, workload_state
from parity_metrics import TOL, check_field

pytestmark = pytest.mark.gpu

W = WORKLOADS["fp64_n2e4_l8"]


def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2111_13072_gb300 import build, imrp
    build.build()
    return torch, imrp


def _oracle_params(p, n):
    return oracle.from_physical(W.R_E_m, W.R_D_m, W.eps_D, W.R_out_m, W.n_e_m3, W.T_e_eV, n, p.l_max,
                                p.dt, drive_kind=p.drive_kind, V_volts=p.V_volts, width_wpe=p.width_wpe,
                                self_image=p.self_image, seed=p.seed)


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_context_and_oracle(prec):
    torch, imrp = _lib()
    stream = torch.cuda.Stream()
    # (n, degree, steps taken before the evaluation, drive): a ragged larger
    # set, a smaller one at another degree, positions and drive of a later step
    # (the Gaussian pulse at t_7), and a small FP32 set whose own tile's image
    # pairs are summed directly
    cases = [(9001, 8, 0, 1, 11), (3001, 16, 0, 1, 12), (2500, 8, 7, 0, 13), (700, 4, 0, 1, 14)]
    for n, L, steps, drive, seed in cases:
        x, v = workload_state(W, N=n)
        x = x[np.random.default_rng(seed).permutation(n)]
        p = imrp.params_from_workload(W, N=n, precision=prec, l_max=L, drive_kind=drive,
                                      V_volts=40.0 if drive == 1 else 300.0)
        with imrp.Sim(p) as sim:
            sim.load(x, v)
            if steps:
                sim.step(steps)
                x, _ = sim.particles()
            E_ref = sim.field()
        xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
        Ed = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        imrp.field_noalloc(p, xd.data_ptr(), n, steps, Ed.data_ptr(), stream.cuda_stream)
        E = Ed.cpu().numpy()
        rel = np.linalg.norm(E - E_ref) / np.linalg.norm(E_ref)
        assert rel < TOL[prec], (n, L, steps, rel)
        op = _oracle_params(p, n)
        Eo = oracle.field_scan(op, x, u=oracle.drive(op, steps))
        check_field(E, Eo, prec, f"noalloc n={n} L={L} step={steps}")


def test_noalloc_allocates_nothing_after_setup():
    torch, imrp = _lib()
    cases = [(2000, 4, 0), (5000, 12, 1), (16384, 16, 0), (100, 1, 1), (4097, 8, 1)]
    bufs = []
    for n, L, prec in cases:  # every caller-owned buffer exists before the set-up
        x, _ = workload_state(W, N=n)
        bufs.append((torch.from_numpy(x).to("cuda"),
                     torch.empty((n, 3), dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()

    def call(k):
        n, L, prec = cases[k]
        p = imrp.params_from_workload(W, N=n, precision=prec, l_max=L, drive_kind=1, V_volts=40.0)
        imrp.field_noalloc(p, bufs[k][0].data_ptr(), n, 0, bufs[k][1].data_ptr())

    call(0)  # set-up on this device (if no earlier call made it)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st0 = {k: v for k, v in torch.cuda.memory_stats().items() if "current" in k}
    E0 = bufs[0][1].cpu().numpy()
    for k in range(1, len(cases)):
        call(k)
    call(0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    st1 = {k: v for k, v in torch.cuda.memory_stats().items() if "current" in k}
    assert free1 == free0, f"free device memory changed by {free1 - free0} bytes"
    assert st1 == st0
    # the shared scratch keeps nothing from one call to the next that matters
    np.testing.assert_array_equal(bufs[0][1].cpu().numpy(), E0)


def test_noalloc_rejects_beyond_limits():
    torch, imrp = _lib()
    p = imrp.params_from_workload(W, N=10)
    xd = torch.ones(20000, 3, dtype=torch.float64, device="cuda") * 1.2
    Ed = torch.empty(20000, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(imrp.IMRPError) as e:
        imrp.field_noalloc(p, xd.data_ptr(), 20000, 0, Ed.data_ptr())
    assert e.value.code == -1
    p24 = imrp.params_from_workload(W, N=10, l_max=24)
    with pytest.raises(imrp.IMRPError):
        imrp.field_noalloc(p24, xd.data_ptr(), 100, 0, Ed.data_ptr())

"""The radius sort (Sec. 3 orders every pair by r_< and r_>; equal radii keep
the storage order) through the public calls, bit for bit.

After a load the storage order is the load order (ids 0..n-1); the first
step sorts it by the radius key and pushes the particles in that order, which
imrp_checkpoint returns. So the ids of a checkpoint after one step must equal
numpy's stable argsort of the keys of the loaded positions, and those of the
next step the stable argsort of the keys of the first step's positions in
their storage order. The key (32 bits of the exact r^2 of the stored position
over [1, r_out^2], include/imrp.h) is recomputed here in integer arithmetic for
FP32 positions and in the library's FP64 expression for FP64 ones, so the
comparison is exact. The cases cover every form of the sort: one CTA, the
top-byte pass with 256 buckets, the 10-bit top pass with 1024 buckets, a
radially narrow shell whose buckets overflow shared memory, exact radius ties,
the four global passes beyond the bucket sort, and contexts that share the GPU
in a batch (several buckets per CTA).
"""
import math

import numpy as np
import pytest

from paper_2111_13072_gb300.inputs import Workload, maxwellian_shell

pytestmark = pytest.mark.gpu

W = Workload("sort", N=1, l_max=2, T_e_eV=3.0, n_e_m3=1e16, drive_kind=2)


@pytest.fixture(scope="module")
def imrp():
    import torch
    assert torch.cuda.is_available(), "these tests need the GPU"
    from paper_2111_13072_gb300 import build, imrp as m
    build.build()
    m.load_library()
    return m


def _umul64hi(a, b):
    """High 64 bits of the 128-bit products of uint64 arrays a and b."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a0, a1 = a & m32, a >> s32
    b0, b1 = b & m32, b >> s32
    p00, p01, p10, p11 = a0 * b0, a0 * b1, a1 * b0, a1 * b1
    mid = (p00 >> s32) + (p01 & m32) + (p10 & m32)
    return p11 + (p01 >> s32) + (p10 >> s32) + (mid >> s32)


def _sq_fx56(v32):
    """floor(v^2 2^56) of float32 values |v| < 8, exactly."""
    u = v32.view(np.uint32).astype(np.uint64)
    e8 = ((u >> np.uint64(23)) & np.uint64(0xFF)).astype(np.int64)
    S = (u & np.uint64(0x7FFFFF)) | np.uint64(0x800000)
    S2 = S * S
    t = 2 * e8 - 244
    left = S2 << np.clip(t, 0, 63).astype(np.uint64)
    right = S2 >> np.clip(-t, 0, 63).astype(np.uint64)
    out = np.where(t >= 0, left, np.where(t <= -64, np.uint64(0), right))
    return np.where(e8 == 0, np.uint64(0), out)


def radius_keys(x, r_out, fp32):
    """The library's radius key of positions x [n, 3] (float64 arrays holding
    the stored values), for a context with outer wall r_out."""
    r2o = r_out * r_out
    if fp32:
        assert r2o < 48.0 and np.all(np.abs(x) < 8.0)
        x32 = x.astype(np.float32)
        assert np.array_equal(x32.astype(np.float64), x)
        R2 = _sq_fx56(x32[:, 0]) + _sq_fx56(x32[:, 1]) + _sq_fx56(x32[:, 2])
        one = np.uint64(1 << 56)
        rout2_fx = np.uint64(int(r2o * 2.0**56))
        ks_fx = np.uint64(int(math.floor(2.0**40 / (r2o - 1.0) + 0.5)))
        hi = _umul64hi(np.where(R2 > one, R2 - one, np.uint64(0)), ks_fx)
        k = np.minimum(hi, np.uint64(0xFFFFFFFF))
        k = np.where(R2 <= one, np.uint64(0), np.where(R2 >= rout2_fx, np.uint64(0xFFFFFFFF), k))
        return k.astype(np.uint32)
    r2 = (x[:, 0] * x[:, 0] + x[:, 1] * x[:, 1]) + x[:, 2] * x[:, 2]
    kf = np.clip((r2 - 1.0) * (4294967296.0 / (r2o - 1.0)), 0.0, 4294967295.0)
    return kf.astype(np.uint32)


def _ties(n, r_out, seed):
    """n positions in groups of 48: the signed permutations of one point, which
    share r^2 exactly in every form of the key; the groups in random order."""
    m = n // 48
    base, _ = maxwellian_shell(m, r_out, 0.0, seed)
    pts = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    pts.append(base[:, perm] * np.array([sx, sy, sz]))
    x = np.concatenate(pts)
    rest, _ = maxwellian_shell(n - x.shape[0], r_out, 0.0, seed + 1)
    x = np.concatenate([x, rest])
    x = x[np.random.default_rng(seed).permutation(n)]
    return np.ascontiguousarray(x)


def _state(kind, n, r_out, seed=5):
    if kind == "uniform":
        x, _ = maxwellian_shell(n, r_out, 0.0, seed)
    elif kind == "narrow":  # all radii within 1e-4: a few top-digit buckets hold everything
        x, _ = maxwellian_shell(n, 1.2001, 0.0, seed, r_in=1.2)
    elif kind == "ties":
        x = _ties(n, r_out, seed)
    else:
        raise ValueError(kind)
    v = np.random.default_rng(seed).standard_normal((n, 3)).astype(np.float32).astype(np.float64) * 0.01
    return x, v


def _check_two_steps(sim, x, fp32, steps=2):
    r_out = sim.info().r_out
    sim.step(1)
    _, _, ids, _ = sim.checkpoint()
    want = np.argsort(radius_keys(x, r_out, fp32), kind="stable").astype(np.uint32)
    np.testing.assert_array_equal(ids, want)
    if steps > 1 and fp32:
        # the second sort: the first step's positions in their storage order
        x1, _, ids1, _ = sim.checkpoint()
        sim.step(1)
        _, _, ids2, _ = sim.checkpoint()
        want2 = ids1[np.argsort(radius_keys(x1, r_out, fp32), kind="stable")]
        np.testing.assert_array_equal(ids2, want2)


CASES = [  # (n, distribution, precision)
    (2000, "uniform", 1),        # one CTA sorts everything
    (100_000, "uniform", 1),     # top byte, 256 buckets
    (100_000, "ties", 0),
    (600_000, "uniform", 1),     # top 10 bits, 1024 buckets
    (600_000, "ties", 1),
    (600_000, "narrow", 1),      # buckets beyond the shared-memory capacity
    (600_000, "uniform", 0),
    (2_000_000, "uniform", 1),   # the benchmark's size
    (2_400_000, "uniform", 1),   # four global passes
]


@pytest.mark.parametrize("n,kind,prec", CASES)
def test_sort_order_is_the_stable_key_order(imrp, n, kind, prec):
    p = imrp.params_from_workload(W, N=n, precision=prec)
    with imrp.Sim(p) as sim:
        x, v = _state(kind, n, sim.info().r_out)
        sim.load(x, v)
        _check_two_steps(sim, x, fp32=prec == 1)


def test_sort_order_in_a_batch(imrp):
    """Contexts stepped together share the GPU: small ones take segments of
    several buckets per CTA; the permutation is the same."""
    sizes = [(600_000, "uniform"), (100_000, "ties"), (20_000, "uniform"), (2_000_000, "uniform")]
    sims, xs = [], []
    try:
        for k, (n, kind) in enumerate(sizes):
            s = imrp.Sim(imrp.params_from_workload(W, N=n, precision=1, seed=k))
            x, v = _state(kind, n, s.info().r_out, seed=11 + k)
            s.load(x, v)
            sims.append(s)
            xs.append(x)
        b = imrp.Batch(sims)
        b.step(1)
        b.sync()
        for s, x in zip(sims, xs):
            _, _, ids, _ = s.checkpoint()
            want = np.argsort(radius_keys(x, s.info().r_out, True), kind="stable").astype(np.uint32)
            np.testing.assert_array_equal(ids, want)
        b.close()
    finally:
        for s in sims:
            s.close()

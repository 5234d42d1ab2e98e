"""The radius-key replication that tests/test_gpu_sort.py compares the GPU sort
against, pinned on the CPU: floor(v^2 2^56) of float32 values against exact
integer arithmetic, the fixed-point key against the FP64 formula
floor((r^2 - 1) / (r_out^2 - 1) 2^32) within one unit, monotonicity in the
exact r^2, and the clamps at the two walls."""
import math
from fractions import Fraction

import numpy as np

from test_gpu_sort import _sq_fx56, radius_keys


def test_square_in_fixed_point_is_exact():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.uniform(-7.9, 7.9, 2000), rng.uniform(-1e-3, 1e-3, 200),
                        np.array([0.0, 1.0, -1.0, 2.0**-40, 7.5])]).astype(np.float32)
    got = _sq_fx56(v)
    for x, g in zip(v.tolist(), got.tolist()):
        exact = math.floor(Fraction(x) ** 2 * 2**56)
        assert g == exact, (x, g, exact)


def test_fixed_point_key_matches_the_fp64_formula():
    rng = np.random.default_rng(4)
    r_out = 1.515
    n = 20000
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = (1.0 + rng.random(n) * (r_out**3 - 1.0)) ** (1.0 / 3.0)
    x = (d * r[:, None]).astype(np.float32).astype(np.float64)
    k32 = radius_keys(x, r_out, True).astype(np.int64)
    k64 = radius_keys(x, r_out, False).astype(np.int64)
    assert np.max(np.abs(k32 - k64)) <= 1
    # monotone in the exact r^2 (FP64 sums of squares of float32 values)
    r2 = (x * x).sum(axis=1)
    o = np.argsort(r2, kind="stable")
    assert np.all(np.diff(k32[o]) >= 0)


def test_keys_clamp_at_the_walls():
    r_out = 1.515
    x = np.array([[1.0, 0.0, 0.0], [0.5, 0.0, 0.0], [r_out, 0.0, 0.0], [2.0, 0.0, 0.0]])
    x = x.astype(np.float32).astype(np.float64)
    for fp32 in (True, False):
        k = radius_keys(x, r_out, fp32)
        assert k[0] == 0 and k[1] == 0
        assert k[3] == 0xFFFFFFFF
        assert k[2] >= 0xFFFFFF00  # at the outer wall, up to float32 rounding of r_out

"""Error metrics of the GPU-against-oracle parity tests.

The tolerances are the method's precision contract for the per-step field E:
1e-5 relative on the FP64 path and 1e-4 on the mixed path (FP32 state,
harmonics and push with FP64 carries), as ||E_gpu - E_orc|| / ||E_orc|| over all
particles. Beside the norm, the per-particle metric
|dE_k| / max(|E_k|, 0.1 E_rms) at its 99.9th percentile keeps a few badly
wrong particles (a tie in the radius order, a particle at a wall, the ragged
last tile) from hiding in the norm. Its bound is ten times the norm bound: the
norm averages the rounding of the ~10^3 terms of every particle over all
particles, and one particle in a thousand may sit an order of magnitude above
that mean (a small field that is the difference of large far- and near-field
parts).
"""
import numpy as np

TOL = {0: 1e-5, 1: 1e-4}
P999 = {0: 1e-4, 1: 1e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def p999(E, Eo):
    mag = np.linalg.norm(Eo, axis=1)
    floor = 0.1 * np.sqrt(np.mean(mag ** 2))
    return float(np.percentile(np.linalg.norm(E - Eo, axis=1) / np.maximum(mag, floor), 99.9))


def check_field(E, Eo, prec, label=""):
    r, p = rel(E, Eo), p999(E, Eo)
    print(f"{label} prec={prec}: ||dE||/||E|| = {r:.3e}, p99.9 = {p:.3e}")
    assert r < TOL[prec]
    assert p < P999[prec]

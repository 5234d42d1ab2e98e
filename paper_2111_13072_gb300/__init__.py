"""GB300-native spectral kinetic simulation of the ideal Multipole Resonance Probe.

The hot path (radius sort, moment scans, field gather, leapfrog push, walls,
Q_diff tally, spectrum) runs in hand-written sm_103a CUDA kernels behind the
C ABI declared in include/imrp.h. ``paper_2111_13072_gb300.imrp`` is the thin
ctypes binding; ``paper_2111_13072_gb300.inputs`` draws seeded synthetic inputs.
"""
__all__ = ["imrp", "inputs"]

"""Runs of the FP64 oracle over many seeds, spread over the host cores in
spawned processes (the oracle itself is single-threaded). Test
infrastructure for the statistical spectrum comparison."""
import multiprocessing as mp
import os

import numpy as np


def _one(args):
    import oracle
    from paper_2111_13072_gb300.inputs import workload_state
    w, nsteps = args
    x, v = workload_state(w)
    op = oracle.from_physical(w.R_E_m, w.R_D_m, w.eps_D, w.R_out_m, w.n_e_m3, w.T_e_eV, w.N, w.l_max, w.dt,
                              drive_kind=w.drive_kind, V_volts=w.V_volts, width_wpe=w.width_wpe, seed=w.seed)
    _, _, q, u, _ = oracle.run(op, x, v, nsteps)
    return q, u


def run_many(workloads, nsteps):
    """(q, u) series of the oracle's run of each workload, in order."""
    try:
        nc = len(os.sched_getaffinity(0))
    except AttributeError:
        nc = os.cpu_count() or 1
    nc = max(1, min(nc, len(workloads)))
    with mp.get_context("spawn").Pool(nc) as pool:
        res = pool.map(_one, [(w, nsteps) for w in workloads])
    return [(np.asarray(q), np.asarray(u)) for q, u in res]

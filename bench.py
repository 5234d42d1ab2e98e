#!/usr/bin/env python
"""Throughput of the IMRP hot path (radius sort, moment scans, field gather,
leapfrog push, walls, Q_diff tally) in particle-steps/s.

Default workload: N = 2e6 electron super-particles, l_max = 16, mixed precision
(FP32 state, harmonics and push; FP64 scan carries), T_e = 3 eV,
n_e = 1e16 m^-3, R_E = 4 mm, R_D = 5 mm, eps_D = 4, R_out = R_D + 20 lambda_D,
dt = 0.05/omega_pe, Gaussian 1 V pulse; seeded synthetic Maxwellian shell.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the instances do not exchange data); value = all particle-steps / max time.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at N=2e6,l_max=16 (mixed vs FP64); served spectra p50/p99"
UNIT = "particle-steps/s"
BUCKET_SORT_SINGLE_N = 3072  # the library sorts up to this many keys in 1 launch,
BUCKET_SORT_MAX_N = 2250000  # up to this many in 4, more in 12


def sort_launches(n):
    """Kernel launches of one radius sort of n keys: one CTA for all of a small
    array; up to BUCKET_SORT_MAX_N keys the top-byte pass (histogram, row scan,
    scatter) and the per-bucket kernel; four such passes (12 launches) beyond."""
    if n <= 1:
        return 0
    if n <= BUCKET_SORT_SINGLE_N:
        return 1
    return 4 if n <= BUCKET_SORT_MAX_N else 12


def step_launches(n):
    """Kernel launches of one step of one instance: sort, reorder, moments, tile
    scan, two group-scan kernels, finalize, field."""
    return sort_launches(n) + 7


def workload_desc(w):
    return (f"{w.name}: N={w.N}, l_max={w.l_max}, T_e={w.T_e_eV} eV, n_e={w.n_e_m3:g} m^-3, "
            f"R_E={w.R_E_m*1e3:g} mm, R_D={w.R_D_m*1e3:g} mm, eps_D={w.eps_D}, "
            f"R_out=R_D+{w.outer_debye:g} lambda_D, dt={w.dt}/omega_pe, Gaussian {w.V_volts} V pulse "
            f"(width {w.width_wpe}), {'mixed (FP32 state/harmonics/push, FP64 carries)' if w.precision else 'FP64'}")


def field_flops_per_particle(L):
    """FP32 flops of one particle in the field kernel (FMA = 2), counted from the
    code as it executes: gradient expansions of degree 1..L+1 (Is) and 0..L-1
    (Rs), column by column. A column m >= 1 is the complex diagonal times a
    real recurrence: 16 flops per entry after the first (the scaled three-term
    step, six FMAs of the contraction), 12 for the column's product with the
    diagonal, 8 for the diagonal step; the real column m = 0 takes 10 per entry
    (6 for the Rs entry l = 0) and 6 at its end. 16 pair evaluations of the
    in-tile direct near field, each 13 flops per degree step of the scaled
    Legendre recurrences (10 for the first) plus 57 for the pair geometry and
    the gradient at both ends; 50 for the l = 0 term, the push and the walls,
    and 2 L for the removal of the particle's own image."""
    far = 10 * (L + 1) + 6 + sum(16 * (L + 1 - m) + 12 + 8 for m in range(1, L + 2))
    far += 6 + 10 * (L - 1) + 6 + sum(16 * (L - m - 1) + 12 + 8 for m in range(1, L))
    near = 16 * (13 * (L - 1) - (3 if L >= 2 else 0) + 57)
    return far + near + 50 + 2 * L


def kernel_hash():
    """Hash of the sources the field kernel is built from (its template, the
    device helpers and the per-degree instantiation units): a DRAM traffic
    record under profiles/ applies only while these are unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2111_13072_gb300", "csrc")
    files = ["imrp_kernels.cuh", "imrp_device.cuh", "imrp_inst.cuh"] + sorted(
        os.path.basename(f) for f in glob.glob(os.path.join(csrc, "imrp_inst_*.cu")))
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def field_traffic(workload_name):
    """DRAM bytes per field launch of this workload from profiles/field_traffic.json
    (an ncu capture), or None unless it was taken of the current kernel sources."""
    tf = os.path.join(ROOT, "profiles", "field_traffic.json")
    if not os.path.exists(tf):
        return None
    try:
        recs = json.load(open(tf))
        for rec in recs if isinstance(recs, list) else [recs]:
            if rec.get("kernel_hash") == kernel_hash() and rec.get("workload") == workload_name:
                return rec.get("dram_bytes_per_launch")
    except Exception:
        return None
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for k, nm in enumerate(names):
                    if r[4 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_sample(w, n, seed, L=None):
    import oracle
    from paper_2111_13072_gb300.inputs import Workload, workload_state
    L = w.l_max if L is None else L
    ws = Workload(w.name, N=n, l_max=L, T_e_eV=w.T_e_eV, n_e_m3=w.n_e_m3, R_E_m=w.R_E_m, R_D_m=w.R_D_m,
                  eps_D=w.eps_D, outer_debye=w.outer_debye, outer_R=w.outer_R, dt=w.dt,
                  drive_kind=w.drive_kind, V_volts=w.V_volts, width_wpe=w.width_wpe, seed=seed)
    p = oracle.from_physical(w.R_E_m, w.R_D_m, w.eps_D, w.R_out_m, w.n_e_m3, w.T_e_eV, n, L, w.dt,
                             drive_kind=w.drive_kind, V_volts=w.V_volts, width_wpe=w.width_wpe, seed=seed)
    x, v = workload_state(ws)
    return p, x, v


def _oracle_timed_run(args):
    """One worker of the host baseline: `warmup` untimed then `steps` timed
    oracle steps on its own sample; returns the timed seconds."""
    w, n, seed, warmup, steps = args
    import oracle
    p, x, v = _oracle_sample(w, n, seed)
    if warmup:
        x, v, _, _, _ = oracle.run(p, x, v, warmup)
    t = time.perf_counter()
    oracle.run(p, x, v, steps, step0=warmup, first_half_kick=warmup == 0)
    return time.perf_counter() - t


def _oracle_per_particle_step(w):
    import oracle
    p, x, v = _oracle_sample(w, 1000, w.seed)
    t = time.perf_counter()
    oracle.run(p, x, v, 1)
    return (time.perf_counter() - t) / 1000.0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(w, budget_s=15.0):
    """The FP64 oracle (radius-ordered scan evaluator, leapfrog, walls) as it
    stands, on bounded samples of the same workload (same geometry, density,
    temperature and l_max): once on one host core, and as one independent
    sample per core on all host cores (spawned processes, the oracle itself
    is single-threaded); particle-steps/s = all particles x steps / wall time."""
    import multiprocessing as mp
    per = _oracle_per_particle_step(w)
    ns = int(max(1000, min(20000, budget_s / 10.0 / per)))
    steps = max(1, int(budget_s / (per * ns)))
    t1 = _oracle_timed_run((w, ns, w.seed, 0, steps))
    single = {"value": ns * steps / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
              "sample": f"{ns} particles x {steps} steps of the same workload (l_max={w.l_max}), "
                        f"scan evaluator, {t1:.1f} s"}
    nc = host_cores()
    with mp.get_context("spawn").Pool(nc) as pool:
        pool.map(_oracle_per_particle_step, [w] * nc)  # start-up and import outside the timing
        t = time.perf_counter()
        pool.map(_oracle_timed_run, [(w, ns, w.seed + 1000 * (k + 1), 0, steps) for k in range(nc)])
        tn = time.perf_counter() - t
    return {"value": nc * ns * steps / tn, "unit": UNIT, "cores": nc, "kind": "oracle",
            "sample": f"{nc} independent samples (one per host core, spawned processes) of {ns} particles "
                      f"x {steps} steps of the same workload (l_max={w.l_max}), scan evaluator, {tn:.1f} s",
            "single_core": single}


def _brute_samples(args):
    w, N, idx = args
    import oracle
    from paper_2111_13072_gb300.inputs import workload_state
    x, _ = workload_state(w)
    p = oracle.from_physical(w.R_E_m, w.R_D_m, w.eps_D, w.R_out_m, w.n_e_m3, w.T_e_eV, N, w.l_max, w.dt,
                             drive_kind=w.drive_kind, V_volts=w.V_volts, width_wpe=w.width_wpe, seed=w.seed)
    return oracle.field_brute(p, x, u=oracle.drive(p, 0), sample=idx)


def oracle_error(w, fields, n_sample=32):
    """The FP64 oracle's error of each precision's field at the workload itself
    (step 0, the loaded state): sampled particles (the 3 innermost, the 3
    outermost and random ones) against the oracle's direct pair sum (the
    definition), spread over the host cores. fields: {name: E [N,3]}."""
    import multiprocessing as mp
    from paper_2111_13072_gb300.inputs import workload_state
    x, _ = workload_state(w)
    order = np.argsort(np.linalg.norm(x, axis=1))
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([order[:3], order[-3:], rng.choice(w.N, n_sample - 6, replace=False)]))
    nc = min(host_cores(), len(idx))
    parts = [idx[k::nc] for k in range(nc)]
    with mp.get_context("spawn").Pool(nc) as pool:
        res = pool.map(_brute_samples, [(w, w.N, part) for part in parts])
    Eo = np.zeros((len(idx), 3))
    pos = {int(i): k for k, i in enumerate(idx)}
    for part, E in zip(parts, res):
        for i, e in zip(part, E):
            Eo[pos[int(i)]] = e
    out = {}
    mag = np.linalg.norm(Eo, axis=1)
    for name, E in fields.items():
        d = np.linalg.norm(E[idx] - Eo, axis=1)
        out[name] = {"norm": float(np.linalg.norm(E[idx] - Eo) / np.linalg.norm(Eo)),
                     "max_per_particle": float(np.max(d / mag)),
                     "median_per_particle": float(np.median(d / mag))}
    out["sample"] = (f"{len(idx)} particles of the loaded state (3 innermost, 3 outermost, the rest random) "
                     f"against the oracle's direct pair sum, {nc} host processes")
    return out


def ensemble_measure(steps, warmup, autotune=True, n_instances=64, stream=None):
    """The 64-instance ensemble (N log-uniform in [1e4, 1e6], T_e in [0.5, 5] eV,
    n_e log-uniform in [1e14, 1e17] m^-3, l_max in {8, 12, 16}, mixed precision),
    stepped as one batch; device time with CUDA events on the batch stream."""
    import torch
    from paper_2111_13072_gb300 import imrp
    from paper_2111_13072_gb300.inputs import workload_state
    from paper_2111_13072_gb300.serve import ensemble_workloads
    ws = ensemble_workloads(n_instances)
    sims = []
    for w in ws:
        s = imrp.Sim(imrp.params_from_workload(w))
        x, v = workload_state(w)
        s.load(x, v)
        if autotune:
            s.autotune()
        sims.append(s)
    stream = stream or torch.cuda.Stream()
    with imrp.Batch(sims) as b:
        b.set_stream(stream.cuda_stream)
        if autotune:
            b.autotune()  # the CTA size of each batched field launch
        b.step(warmup)
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        b.sync()
        ms = e0.elapsed_time(e1)
    ntot = sum(w.N for w in ws)
    for s in sims:
        s.close()
    # per context: sort, reorder, tile scan, two group-scan kernels, finalize;
    # per degree and precision: one moments and one field launch
    launches = sum(sort_launches(w.N) + 5 for w in ws) + 2 * len({(w.precision, w.l_max) for w in ws})
    return {"value": ntot * steps / (ms / 1e3), "unit": UNIT, "instances": n_instances,
            "gpu_launches_per_step": launches,
            "particles": ntot, "steps": steps, "ms_per_step": ms / steps, "autotuned": autotune,
            "workload": "64 instances, N log-uniform [1e4,1e6], T_e U[0.5,5] eV, n_e log-U[1e14,1e17], "
                        "l_max in {8,12,16}, mixed precision, one captured graph per step pair, "
                        "one moments and one field launch per degree"}


def ensemble_compare(steps, warmup):
    """The 64-instance ensemble with the launch shapes the library picks at
    creation and with the autotuners' choices (imrp_autotune per context for
    its scans, imrp_batch_autotune for the batched field launches), each timed."""
    plain = ensemble_measure(steps, warmup, autotune=False)
    tuned = ensemble_measure(steps, warmup, autotune=True)
    tuned["default_shapes"] = {"value": plain["value"], "ms_per_step": plain["ms_per_step"]}
    tuned["speedup_over_default"] = tuned["value"] / plain["value"]
    return tuned


def serving_measure(n_requests, steps, rate=20.0):
    """Continuous-batching service: Poisson arrivals at `rate` of spectrum
    requests (N log-uniform in [1e5, 4e6], T_e in [0.5, 5] eV, n_e log-uniform
    in [1e14, 1e17] m^-3, l_max in {8, 16}, `steps` steps each) over a bounded
    horizon of n_requests; latency = completion (spectrum ready) - arrival.
    The offered load is rate x the mean particle-steps of a request; the
    sustained throughput is all particle-steps over the span from the first
    arrival to the last completion; the highest arrival rate the device
    sustains (at which the queue, and so p99, stays bounded) is the
    sustained throughput over the mean request."""
    from paper_2111_13072_gb300.serve import SpectrumServer, serving_requests
    reqs = serving_requests(n_requests, rate=rate, steps=steps)
    srv = SpectrumServer(chunk=250)
    t0 = time.perf_counter()
    res = srv.serve(reqs, realtime=True)
    span = time.perf_counter() - t0
    lat = np.array([r.latency for r in res])
    work = np.array([r.workload.N * r.steps for r in reqs], dtype=np.float64)
    sustained = float(work.sum() / span)
    return {"requests": n_requests, "steps_per_request": steps, "rate_req_per_s": rate,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "spectra_per_s": n_requests / span, "particle_steps_per_s": sustained,
            "offered_particle_steps_per_s": float(rate * work.mean()),
            "max_sustainable_rate_req_per_s": float(sustained / work.mean()),
            "errors": int(sum(r.error is not None for r in res)),
            "max_active": srv.stats["max_active"], "peak_bytes": srv.stats["peak_bytes"],
            "span_s": span,
            "workload": f"Poisson arrivals at {rate:g} req/s, {n_requests} requests of {steps} steps, "
                        "N log-uniform [1e5,4e6], T_e U[0.5,5] eV, n_e log-U[1e14,1e17], "
                        "l_max in {8,16}, mixed precision"}


ARGON_MASS_RATIO = 39.948 * 1822.888486  # m_i / m_e; the paper names no gas


def _paired_response_fit(T, nu_coll, N, seeds, steps, t_win, sheath=False):
    """Kick-minus-no-kick Q_diff on the paper's case, averaged over seeds, and
    the fit a e^{-bt} sin(ct + phi) over 0 <= t <= t_win of the mean and of
    the two halves of the seeds. sheath: start from the floating equilibrium
    (App. D; immobile ions of its profile, its surface charge, electrons drawn
    from its Boltzmann density) instead of the uniform shell."""
    from paper_2111_13072_gb300 import imrp
    from paper_2111_13072_gb300.inputs import paper_variant, radial_profile_shell, workload_state
    dqs = []
    eq = None
    for seed in range(seeds):
        w = paper_variant(T, N=N, steps=steps, seed=seed)
        if sheath:
            if eq is None:
                eq = imrp.sheath_solve(w.sigma_v, ARGON_MASS_RATIO, w.r_out, 4097)
            x, v = radial_profile_shell(N, eq["r"], eq["q_elec"], w.sigma_v, seed=seed)
        else:
            x, v = workload_state(w)
        series = {}
        for kind in (w.drive_kind, 2):  # the kick, then no drive
            with imrp.Sim(imrp.params_from_workload(w, drive_kind=kind, nu_coll=nu_coll)) as sim:
                if sheath:
                    sim.set_ion_profile(eq["q_ion"], eq["q_elec"][-1], eq["q_s"])
                sim.load(x, v)
                sim.step_async(steps)
                sim.sync()
                series[kind] = sim.qdiff()
        dqs.append(series[w.drive_kind][0] - series[2][0])
        u = series[w.drive_kind][1]

    def fit(dq):
        om, re, im = imrp.admittance(dq, u, w.dt, 0.5 * w.dt, 1000, 2.0)
        w0 = float(om[int(np.argmax(re))])
        try:
            return imrp.fit_damped_sine(dq, w.dt, 0.0, t_win, w0, 0.05)
        except imrp.IMRPError:
            return np.full(4, np.nan)

    a, b, c, ph = fit(np.mean(dqs, axis=0))
    h = len(dqs) // 2
    halves = [2.0 * float(fit(np.mean(dqs[:h], axis=0))[1]), 2.0 * float(fit(np.mean(dqs[h:], axis=0))[1])]
    r = {"fit_a_b_c_phi": [float(a), float(b), float(c), float(ph)], "nu_eff": 2.0 * float(b),
         "nu_eff_halves": halves, "drude_eta": float(np.hypot(b, c))}
    if eq is not None:
        r["sheath"] = {"rhat": float(eq["rhat"]), "psi_wall": float(eq["psi_wall"]),
                       "q_s": float(eq["q_s"])}
    return r, w


def drude_measure(temps=(2.0, 3.0, 5.0), N=500000, steps=3000, seeds=4, t_win=30.0, nus=(0.1, 0.2),
                  sheath=False):
    """The paper's temperature diagnostic (Sec. 4) on its own case (R = 4 mm,
    1 mm dielectric, n = 1e15 m^-3, 1 < r < 10, l <= 1 / m = 0 kernel, one
    kick u_asy = 1, dt = 0.01) with the uniform Maxwellian shell in place of
    its sheath. The shell is not an equilibrium and its spontaneous Q_diff
    fluctuations are ten times the kick's response, so for each T_e and seed
    a correlated pair of runs from one state, with and without the kick, is
    differenced (the fluctuations, the same in both until the trajectories part
    after a few plasma periods, cancel) and the differences of `seeds` states
    are averaged. As in the paper, the response is fitted with
    a e^{-bt} sin(ct + phi) over 0 <= t <= t_win; its transform is the Drude
    dipole term with nu_eff = 2 b and eta = sqrt(b^2 + c^2), and
    K = nu_eff R / lambda_D. The paper, with its sheath, reports nu_eff in
    {0.105, 0.128, 0.167} and K = 1.264. Then, at 3 eV, electron-neutral
    collisions at the rates `nus`: the Drude model adds nu to the damping.
    sheath: every run starts from the floating equilibrium of App. D instead
    (argon ions, immobile)."""
    import torch
    from paper_2111_13072_gb300 import imrp
    out, coll = [], []
    t0 = time.perf_counter()
    for T in temps:
        r, w = _paired_response_fit(T, 0.0, N, seeds, steps, t_win, sheath)
        nu = r["nu_eff"]
        r.update({"T_e_eV": T, "K": imrp.drude_k(nu, T, w.R_D_m, w.n_e_m3) if nu > 0 else None})
        out.append(r)
    for nc in nus:
        r, w = _paired_response_fit(3.0, nc, N, seeds, steps, t_win, sheath)
        r.update({"T_e_eV": 3.0, "nu_coll": nc})
        coll.append(r)
    torch.cuda.synchronize()
    Ks = [r["K"] for r in out if r["K"] is not None]
    return {"runs": out, "K_mean": float(np.mean(Ks)) if Ks else None, "collisions": coll, "N": N,
            "steps": steps, "seeds": seeds, "t_window": t_win, "seconds": time.perf_counter() - t0,
            "workload": "paper's case: R=4 mm, R_E=3 mm, eps_D=4, n=1e15 m^-3, 1<r<10, l_max=1 m=0 kernel, "
                        "kick u_asy=1, dt=0.01, "
                        + ("floating sheath equilibrium (App. D, argon, immobile ions)" if sheath
                           else "uniform Maxwellian shell (no sheath)")
                        + ", mixed precision; kick minus no-kick runs from the same state, mean over seeds",
            "paper": {"nu_eff": [0.105, 0.128, 0.167], "K": 1.264}}


def run_reference(args, w):
    """--impl reference: the FP64 CPU oracle as the reference arm, on all host
    cores (one independent sample of the workload per core, spawned processes;
    the timed steps of the slowest worker set the time)."""
    import multiprocessing as mp
    per = _oracle_per_particle_step(w)
    total_budget = 90.0
    ns = int(max(200, min(20000, total_budget / (args.steps + args.warmup) / per)))
    nc = host_cores()
    with mp.get_context("spawn").Pool(nc) as pool:
        pool.map(_oracle_per_particle_step, [w] * nc)
        times = pool.map(_oracle_timed_run,
                         [(w, ns, w.seed + 1000 * k, args.warmup, args.steps) for k in range(nc)])
    dt = max(times)
    val = nc * ns * args.steps / dt
    sample = (f"{nc} independent samples (one per host core) of {ns} particles per step "
              f"(same workload, l_max={w.l_max}), scan evaluator, FP64")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_desc(w), "sample_particles": ns,
                       "parallelism": f"host, {nc} cores (independent samples)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": nc, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sub_config(name, steps, warmup, nprof, peak_tflops, stream):
    """Another single-instance workload, timed like the main one (graph-replayed
    steps, CUDA events on the context's stream) with its per-stage device time
    and the field kernel's roofline fraction."""
    import torch
    from paper_2111_13072_gb300 import imrp
    from paper_2111_13072_gb300.inputs import WORKLOADS, workload_state
    w = WORKLOADS[name]
    x, v = workload_state(w)
    with imrp.Sim(imrp.params_from_workload(w)) as sim:
        sim.set_stream(stream.cuda_stream)
        sim.load(x, v)
        sim.step_async(warmup)
        sim.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step_async(steps)
        e1.record(stream)
        sim.sync()
        ms = e0.elapsed_time(e1)
        stages = sim.profile_steps(nprof)
    field_ms = stages["field"] / nprof
    K = (w.l_max + 1) ** 2
    out = {"workload": workload_desc(w), "value": w.N * steps / (ms / 1e3), "unit": UNIT, "steps": steps,
           "warmup": warmup, "ms_per_step": ms / steps, "dtype": "f32" if w.precision else "f64",
           "stage_ms_per_step": {k: v / nprof for k, v in stages.items()},
           "gpu_launches": step_launches(w.N) * steps}
    if w.precision:
        ach = field_flops_per_particle(w.l_max) * w.N / (field_ms / 1e3) / 1e12
        ach24 = 24.0 * K * w.N / (field_ms / 1e3) / 1e12
        out["roofline"] = {"bound": "alu", "kernel": "k_field (gather+push)", "achieved": ach,
                           "peak": peak_tflops, "unit": "TFLOP/s", "frac": ach / peak_tflops,
                           "frac_24K_model": ach24 / peak_tflops,
                           "flops_per_particle": field_flops_per_particle(w.l_max),
                           "traffic": field_traffic(w.name)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed_n2e6_l16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-sub-configs", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="bounded horizon of the serving measurement (requests of 5000 steps)")
    ap.add_argument("--no-oracle-err", action="store_true")
    ap.add_argument("--drude", action="store_true",
                    help="also run the T_e sweep of the temperature diagnostic on the paper's case")
    ap.add_argument("--drude-n", type=int, default=500000)
    ap.add_argument("--drude-seeds", type=int, default=4)
    ap.add_argument("--drude-sheath", action="store_true",
                    help="start the --drude runs from the floating sheath equilibrium (App. D)")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2111_13072_gb300.inputs import WORKLOADS, workload_state
    if args.workload in ("ensemble64", "serving"):
        import torch
        torch.cuda.set_device(local)
        from paper_2111_13072_gb300 import build
        build.build()
        if args.workload == "ensemble64":
            with ClockSampler(local) as clk:
                r = ensemble_measure(args.steps, args.warmup)
            line = {"metric": "particle-steps/s, 64-instance batched ensemble", "value": r["value"],
                    "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                    "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                    "config": {"workload": r["workload"], "particles": r["particles"]},
                    "clocks": clk.summary(), "gpu_launches": r["gpu_launches_per_step"] * args.steps}
        else:
            r = serving_measure(max(4, args.steps // 50), args.steps)
            line = {"metric": "served spectra p50/p99 latency", "value": r["p50_s"], "unit": "s",
                    "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": 0,
                    "p99_s": r["p99_s"], "spectra_per_s": r["spectra_per_s"], "data": "synthetic",
                    "dtype": "f32", "config": r, "vs_baseline": None, "scaling": "weak"}
        print(json.dumps(line), flush=True)
        return
    w = WORKLOADS[args.workload]

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2111_13072_gb300 import build, imrp
    from paper_2111_13072_gb300.replicas import max_over_ranks, rank_seed, throughput
    build.build()
    x, v = workload_state(w)
    p = imrp.params_from_workload(w, seed=rank_seed(w.seed, rank))
    sim = imrp.Sim(p)
    stream = torch.cuda.Stream()
    sim.set_stream(stream.cuda_stream)
    sim.load(x, v)
    # the library's autotuner (field-only passes, the state does not advance):
    # the field CTA size and the group-scan segment length for this instance
    tuned = sim.autotune()
    sim.step_async(args.warmup)
    sim.sync()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        sim.step_async(args.steps)
        e1.record(stream)
        sim.sync()
        barrier()
    ms = max_over_ranks([e0.elapsed_time(e1)], dist, "cuda")[0]
    N = w.N
    value = throughput(N, args.steps, world, ms / 1e3)
    clocks = clk.summary()

    # per-stage device time (real steps launched one by one, CUDA events)
    nprof = min(args.steps, 50)
    stages = sim.profile_steps(nprof)
    field_ms = stages["field"] / nprof
    K = (w.l_max + 1) ** 2
    flops_per_launch = float(field_flops_per_particle(w.l_max)) * N  # recounted model, times N
    achieved = flops_per_launch / (field_ms / 1e3) / 1e12
    # coarse per-particle model: 24 K flops (harmonics, scans, three contractions), K = (L+1)^2
    achieved_24k = 24.0 * K * N / (field_ms / 1e3) / 1e12
    sm_mhz = clocks["sm_mhz"] or 2070.0
    # measured FP32 FMA throughput of this device (imrp_fp32_peak: independent
    # FMA chains on every SM, the SM count read from the device)
    peak, n_sm = imrp.fp32_peak()
    peak_derived = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
    traffic = field_traffic(w.name)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_field (gather+push)",
                "flops_per_particle": field_flops_per_particle(w.l_max),
                "achieved_24K_model": achieved_24k, "frac_24K_model": achieved_24k / peak,
                "peak_basis": "measured (imrp_fp32_peak: FFMA chains on all SMs)",
                "peak_derived": peak_derived,
                "peak_derived_basis": f"{n_sm} SMs x 128 FP32 FMA/clk x 2 x median SM clock {sm_mhz:.0f} MHz",
                "stage_ms_per_step": {k: v / nprof for k, v in stages.items()}}

    # end to end through the public API with host buffers (pinned): every step
    # loads the state from the host (H2D, 48 B per particle), takes one step
    # and reads its Q_diff back (D2H). Streamed form (the value): the calls are
    # queued (imrp_load_particles_async / imrp_step_async /
    # imrp_copy_qdiff_async), so the copy of step k+1's inputs runs on the copy
    # engine while step k computes; one synchronisation at the end. Blocking
    # form (blocking_value): imrp_load_particles + imrp_step, each waiting.
    xh = torch.from_numpy(x).pin_memory()
    vh = torch.from_numpy(v).pin_memory()
    ne = max(3, min(args.steps, 50))
    qh = torch.zeros(ne, dtype=torch.float64).pin_memory()
    sim.load_async_ptr(xh.data_ptr(), vh.data_ptr(), N)
    sim.step_async(1)
    sim.copy_qdiff_async(0, 1, qh.data_ptr())
    sim.sync()
    barrier()
    t0 = time.perf_counter()
    for i in range(ne):
        sim.load_async_ptr(xh.data_ptr(), vh.data_ptr(), N)
        sim.step_async(1)
        sim.copy_qdiff_async(0, 1, qh[i:].data_ptr())
    sim.sync()
    barrier()
    te = time.perf_counter() - t0
    assert np.all(np.isfinite(qh.numpy()))
    qb = torch.zeros(1, dtype=torch.float64).pin_memory()
    sim.load_ptr(xh.data_ptr(), vh.data_ptr(), N)
    sim.step_ptr(1, qb.data_ptr())
    barrier()
    tb0 = time.perf_counter()
    for _ in range(ne):
        sim.load_ptr(xh.data_ptr(), vh.data_ptr(), N)
        sim.step_ptr(1, qb.data_ptr())
    barrier()
    tb = time.perf_counter() - tb0
    te, tb = max_over_ranks([te, tb], dist, "cuda")
    e2e = {"value": throughput(N, ne, world, te), "unit": UNIT, "h2d_bytes_per_step": 48 * N,
           "d2h_bytes_per_step": 8, "steps": ne, "mode": "streamed (H2D of step k+1 overlaps step k)",
           "blocking_value": throughput(N, ne, world, tb)}

    # the field of each precision at the loaded state, for the oracle's error
    sim.load(x, v)
    fields = {"mixed": sim.field()}
    fp64 = None
    if not args.no_fp64:
        p64 = imrp.params_from_workload(w, precision=0, seed=rank_seed(w.seed, rank))
        with imrp.Sim(p64) as s64:
            s64.set_stream(stream.cuda_stream)
            s64.load(x, v)
            fields["fp64"] = s64.field()
            s64.step_async(3)
            s64.sync()
            k64 = 6
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            s64.step_async(k64)
            f1.record(stream)
            s64.sync()
            fp64 = {"value": N * k64 / (f0.elapsed_time(f1) / 1e3), "unit": UNIT, "steps": k64,
                    "note": "plain FP64 GPU path, same workload"}
    sim.close()

    subs = {}
    if not args.no_sub_configs:
        subs["mixed_n1.6e7_l24"] = sub_config("mixed_n1.6e7_l24", 10, 3, 3, peak, stream)
        subs["fp64_n2e4_l8"] = sub_config("fp64_n2e4_l8", 400, 10, 20, peak, stream)

    serving = None if (args.no_serving or rank != 0) else serving_measure(args.serve_requests, 5000)
    ensemble = None if args.no_ensemble else ensemble_compare(200, 4)
    drude = (drude_measure(N=args.drude_n, seeds=args.drude_seeds, sheath=args.drude_sheath)
             if (args.drude and rank == 0) else None)

    cpu = None
    oerr = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    if rank == 0 and not args.no_oracle_err:
        oerr = oracle_error(w, fields)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if w.precision else "f64",
                "data": "synthetic",
                "config": {"workload": workload_desc(w), "N": N, "l_max": w.l_max,
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                           "l2": "inputs larger than L2 (per-step working set > 300 MB)",
                           "autotuned": {"warps_per_cta": tuned[0], "groups_per_segment": tuned[1]}},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": step_launches(N) * args.steps, "clocks": clocks, "fp64_gpu": fp64,
                "oracle_err": oerr, "configs": subs, "serving": serving, "ensemble": ensemble,
                "drude": drude}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

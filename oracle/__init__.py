"""FP64 CPU oracle for the spectral kinetic IMRP hot path (arXiv 2111.13072).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
this package. The product library never imports it, and it imports nothing
from the product package: the two share no code.

The numerical core is plain C in ``imrp_oracle.c`` (built with gcc into
``oracle/_build``); this module holds the ctypes glue, the conversion from
physical to dimensionless parameters (Sec. 4), and the spectrum analysis
(Sec. 4: admittance from the Fourier transform of Q_diff, the damped-sine fit).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SRC = os.path.join(_HERE, "imrp_oracle.c")

# CODATA 2018 constants (SI)
E_CHARGE = 1.602176634e-19
EPS0 = 8.8541878128e-12
M_E = 9.1093837015e-31


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc (plain -O2, IEEE arithmetic)."""
    import platform
    import shutil
    stamp = os.path.join(_BUILD, "MACHINE")
    if os.path.isdir(_BUILD) and (not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine()):
        shutil.rmtree(_BUILD, ignore_errors=True)
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(stamp):
        with open(stamp, "w") as f:
            f.write(platform.machine())
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _FieldParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("eps", ctypes.c_double), ("r_out", ctypes.c_double),
                ("n_tilde", ctypes.c_double), ("n_ion", ctypes.c_double), ("q_s", ctypes.c_double),
                ("L", ctypes.c_int32), ("m0_only", ctypes.c_int32), ("self_image", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("ion_q", ctypes.POINTER(ctypes.c_double)),
                ("ion_n", ctypes.c_int64), ("charge", ctypes.POINTER(ctypes.c_double)),
                ("mass", ctypes.POINTER(ctypes.c_double))]


class _RunParams(ctypes.Structure):
    _fields_ = [("fp", _FieldParams), ("dt", ctypes.c_double), ("drive_kind", ctypes.c_int32),
                ("wall_rule", ctypes.c_int32), ("v_hat", ctypes.c_double), ("sigma", ctypes.c_double),
                ("t0", ctypes.c_double), ("seed", ctypes.c_uint64), ("nu_coll", ctypes.c_double),
                ("sigma_v", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        pd, pi64 = P(d), P(i64)
        _lib.orc_coeffs.argtypes = [i32, d, d, pd, pd, pd, pd, pd, pd]
        _lib.orc_field_brute.argtypes = [P(_FieldParams), i64, pd, pi64, d, i64, pi64, pd]
        _lib.orc_field_scan.argtypes = [P(_FieldParams), i64, pd, pi64, d, pd]
        _lib.orc_green.argtypes = [P(_FieldParams), pd, pd, pd]
        _lib.orc_psi_anti.argtypes = [i32, d, d, pd]
        _lib.orc_psi_anti.restype = d
        _lib.orc_qdiff.argtypes = [P(_FieldParams), i64, pd]
        _lib.orc_qdiff.restype = d
        _lib.orc_energy.argtypes = [P(_FieldParams), i64, pd, pd, pi64, d]
        _lib.orc_energy.restype = d
        _lib.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        _lib.orc_drive.argtypes = [P(_RunParams), i64]
        _lib.orc_drive.restype = d
        _lib.orc_run.argtypes = [P(_RunParams), i64, pd, pd, pi64, i64, i64, i32, i32, pd, pd, pd, pi64]
        _lib.orc_inject_many.argtypes = [P(_RunParams), i64, pd, pd, pi64, i64]
        _lib.orc_collisions.argtypes = [P(_RunParams), i64, pd, pi64, i64]
        _lib.orc_collisions.restype = i64
        _lib.orc_coll_threshold.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib.orc_coll_threshold.restype = ctypes.c_uint32
        _lib.orc_run.restype = i64
    return _lib


def _p(a, ct=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


@dataclass
class Params:
    """Dimensionless problem (Sec. 4 units: R, 1/omega_pe, e, m_e)."""
    d: float
    eps: float
    r_out: float
    n_tilde: float
    n_ion: float
    L: int
    q_s: float = 0.0
    m0_only: int = 0
    self_image: int = 0
    dt: float = 0.05
    drive_kind: int = 2
    wall_rule: int = 0
    v_hat: float = 0.0
    sigma: float = 2.0
    t0: float = 8.0
    seed: int = 0
    nu_coll: float = 0.0
    sigma_v: float = 0.0  # thermal speed of the plasma that wall_rule 2 injects from
    # immobile ions of a radial profile (App. D): ion charge inside
    # r_k = 1 + k (r_out - 1)/(len - 1) in super-particle charges; None: uniform n_ion
    ion_q: np.ndarray = None
    # mobile ions as particles: charge (e) and mass (m_e) per particle, in the
    # order of the arrays passed with these parameters; None: all electrons
    charge: np.ndarray = None
    mass: np.ndarray = None

    def field(self) -> _FieldParams:
        for name in ("ion_q", "charge", "mass"):
            a = getattr(self, name)
            if a is not None:
                setattr(self, name, np.ascontiguousarray(a, dtype=np.float64))
        if self.ion_q is not None:
            assert self.ion_q.ndim == 1 and len(self.ion_q) >= 2
        return _FieldParams(self.d, self.eps, self.r_out, self.n_tilde, self.n_ion, self.q_s,
                            self.L, self.m0_only, self.self_image, 0, _p(self.ion_q),
                            0 if self.ion_q is None else len(self.ion_q), _p(self.charge),
                            _p(self.mass))

    def run(self) -> _RunParams:
        return _RunParams(self.field(), self.dt, self.drive_kind, self.wall_rule, self.v_hat,
                          self.sigma, self.t0, self.seed, self.nu_coll, self.sigma_v)


def from_physical(R_E_m, R_D_m, eps_D, R_out_m, n_e_m3, T_e_eV, N, l_max, dt, drive_kind=0,
                  V_volts=1.0, width_wpe=2.0, t0_wpe=None, wall_rule=0, self_image=0,
                  m0_only=0, seed=0, nu_coll=0.0) -> Params:
    """Converts a physical configuration to the dimensionless problem of Sec. 4.

    Length unit R = R_D (outer radius of the dielectric); d = 1 - R_E/R.
    n~ = N / V_shell is the expected number of super-particles per unit cube
    at density n_inf (Sec. 4). The ion background is uniform and holds N ion
    super-particles (a neutral shell). A voltage V becomes V eps0/(n e R^2).
    The plasma that wall_rule 2 injects has the thermal speed lambda_D omega_pe,
    i.e. lambda_D / R in these units.
    """
    R = R_D_m
    d = 1.0 - R_E_m / R_D_m
    r_out = R_out_m / R
    vsh = 4.0 * np.pi / 3.0 * (r_out ** 3 - 1.0)
    n_tilde = N / vsh
    v_hat = V_volts * EPS0 / (n_e_m3 * E_CHARGE * R * R)
    t0 = 4.0 * width_wpe if t0_wpe is None else t0_wpe
    return Params(d=d, eps=eps_D, r_out=r_out, n_tilde=n_tilde, n_ion=float(N), L=l_max, dt=dt,
                  drive_kind=drive_kind, v_hat=v_hat, sigma=width_wpe, t0=t0, wall_rule=wall_rule,
                  self_image=self_image, m0_only=m0_only, seed=seed, nu_coll=nu_coll,
                  sigma_v=float(debye_length(n_e_m3, T_e_eV) / R))


def debye_length(n_e_m3, T_e_eV):
    return np.sqrt(EPS0 * T_e_eV / (n_e_m3 * E_CHARGE))


def plasma_frequency(n_e_m3):
    return np.sqrt(n_e_m3 * E_CHARGE ** 2 / (EPS0 * M_E))


# ---------------------------------------------------------------- coefficients
def coeffs(L, d, eps):
    """Returns dict of f_l, g_l (App. A), a^D, b^D, b^P (Sec. 3), canti (Psi_anti)."""
    out = {k: np.zeros(L + 1) for k in ("f", "g", "aD", "bD", "bP", "canti")}
    lib().orc_coeffs(L, d, eps, *(_p(out[k]) for k in ("f", "g", "aD", "bD", "bP", "canti")))
    return out


# ---------------------------------------------------------------- fields
def _ids(n, ids):
    return np.arange(n, dtype=np.int64) if ids is None else np.ascontiguousarray(ids, dtype=np.int64)


def field_brute(p: Params, x, u=0.0, ids=None, sample=None):
    """Field by the direct pair sum (the definition). x: [n,3]. sample: indices."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    ids = _ids(n, ids)
    fp = p.field()
    if sample is None:
        E = np.zeros((n, 3))
        lib().orc_field_brute(ctypes.byref(fp), n, _p(x), _p(ids, ctypes.c_int64), u, n, None, _p(E))
    else:
        ks = np.ascontiguousarray(sample, dtype=np.int64)
        E = np.zeros((ks.size, 3))
        lib().orc_field_brute(ctypes.byref(fp), n, _p(x), _p(ids, ctypes.c_int64), u, ks.size,
                              _p(ks, ctypes.c_int64), _p(E))
    return E


def field_scan(p: Params, x, u=0.0, ids=None):
    """Field by the radius-ordered scan (pinned against field_brute)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    ids = _ids(n, ids)
    E = np.zeros((n, 3))
    fp = p.field()
    lib().orc_field_scan(ctypes.byref(fp), n, _p(x), _p(ids, ctypes.c_int64), u, _p(E))
    return E


def green(p: Params, x, xs):
    """G~_L(x, xs) and its gradient in x: returns (G, gradG[3])."""
    out = np.zeros(4)
    fp = p.field()
    lib().orc_green(ctypes.byref(fp), _p(np.ascontiguousarray(x, dtype=np.float64)),
                    _p(np.ascontiguousarray(xs, dtype=np.float64)), _p(out))
    return out[0], out[1:]


def psi_anti(L, d, eps, x):
    return lib().orc_psi_anti(L, d, eps, _p(np.ascontiguousarray(x, dtype=np.float64)))


def qdiff(p: Params, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    fp = p.field()
    return lib().orc_qdiff(ctypes.byref(fp), x.shape[0], _p(x))


def energy(p: Params, x, v, u=0.0, ids=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    ids = _ids(x.shape[0], ids)
    fp = p.field()
    return lib().orc_energy(ctypes.byref(fp), x.shape[0], _p(x), _p(v), _p(ids, ctypes.c_int64), u)


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(o, ctypes.c_uint32))
    return o


def collisions(p: Params, v, step, ids=None):
    """The collision operator alone on velocities v [n,3] at a step index:
    returns (v after, number of collisions)."""
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    ids = _ids(v.shape[0], ids)
    rp = p.run()
    c = lib().orc_collisions(ctypes.byref(rp), v.shape[0], _p(v), _p(ids, ctypes.c_int64), step)
    return v, int(c)


def coll_threshold(nu, dt):
    return int(lib().orc_coll_threshold(nu, dt))


def drive(p: Params, step):
    rp = p.run()
    return lib().orc_drive(ctypes.byref(rp), step)


def run(p: Params, x, v, nsteps, step0=0, first_half_kick=True, evaluator="scan", ids=None,
        surface=False):
    """Leapfrog run; returns (x, v, qdiff[nsteps], uasy[nsteps], wall_hits), and
    with surface=True also Q_S after the last step and the number of probe
    absorptions (wall_rule 2 accrues the absorbed charge into Q_S).

    v on input is synchronous with x when first_half_kick, else the half-step
    velocity; on output it is the half-step velocity v_{n+1/2}.
    """
    x = np.array(x, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    n = x.shape[0]
    ids = _ids(n, ids)
    q = np.zeros(nsteps)
    u = np.zeros(nsteps)
    rp = p.run()
    qs = np.zeros(1)
    nab = np.zeros(1, dtype=np.int64)
    hits = lib().orc_run(ctypes.byref(rp), n, _p(x), _p(v), _p(ids, ctypes.c_int64), step0, nsteps,
                         int(first_half_kick), 0 if evaluator == "brute" else 1, _p(q), _p(u),
                         _p(qs), _p(nab, ctypes.c_int64))
    if surface:
        return x, v, q, u, hits, float(qs[0]), int(nab[0])
    return x, v, q, u, hits


def inject(p: Params, ids, step):
    """The re-injection of wall_rule 2 alone for the given particle ids at a
    step: returns (x [n,3], v [n,3])."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    x = np.zeros((ids.size, 3))
    v = np.zeros((ids.size, 3))
    rp = p.run()
    lib().orc_inject_many(ctypes.byref(rp), ids.size, _p(x), _p(v), _p(ids, ctypes.c_int64), step)
    return x, v


# ---------------------------------------------------------------- spectrum
def kick_weights(nsteps, dt, first_half_kick=True):
    w = np.full(nsteps, dt)
    if first_half_kick and nsteps:
        w[0] = 0.5 * dt
    return w


def spectrum(qd, ua, dt, n_freq, w_max, first_half_kick=True, t_start=0.0):
    """Admittance Y(w) = i w Q^(w) / U^(w) (Sec. 4), by direct DFT sums.

    Q^(w) = dt sum_n (Q_n - Q_0) e^{-i w t_n}; U^(w) = sum_n w_n u_n e^{-i w t_n}
    with w_n the kick weight of step n. Frequencies w_j = (j+1) w_max / n_freq.
    Returns (omega, Y, w_res, dw): w_res = argmax Re Y (parabolic refinement),
    dw = full width at half maximum of Re Y around it.
    """
    qd = np.asarray(qd, dtype=np.float64)
    ua = np.asarray(ua, dtype=np.float64)
    ns = qd.size
    t = t_start + dt * np.arange(ns)
    w = kick_weights(ns, dt, first_half_kick)
    omega = (np.arange(n_freq) + 1.0) * (w_max / n_freq)
    ph = np.exp(-1j * np.outer(omega, t))
    Q = dt * ph @ (qd - qd[0])
    U = ph @ (w * ua)
    Y = 1j * omega * Q / U
    w_res, dw = peak_and_fwhm(omega, Y.real)
    return omega, Y, w_res, dw


def peak_and_fwhm(omega, re):
    j = int(np.argmax(re))
    if 0 < j < len(re) - 1:
        y0, y1, y2 = re[j - 1], re[j], re[j + 1]
        den = y0 - 2 * y1 + y2
        off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
        w_res = omega[j] + off * (omega[1] - omega[0])
    else:
        w_res = omega[j]
    half = 0.5 * re[j]
    lo = j
    while lo > 0 and re[lo] > half:
        lo -= 1
    hi = j
    while hi < len(re) - 1 and re[hi] > half:
        hi += 1

    def cross(a, b):
        if re[a] == re[b]:
            return omega[a]
        return omega[a] + (half - re[a]) * (omega[b] - omega[a]) / (re[b] - re[a])

    w_lo = cross(lo, lo + 1) if re[lo] <= half else omega[lo]
    w_hi = cross(hi - 1, hi) if re[hi] <= half else omega[hi]
    return float(w_res), float(w_hi - w_lo)


def fit_damped_sine(qd, dt, t_fit, w0, b0, t_start=0.0):
    """Least-squares fit of a e^{-b tau} sin(c tau + phi), tau = t - t_fit (Sec. 4, s = 1)."""
    from scipy.optimize import curve_fit
    qd = np.asarray(qd, dtype=np.float64)
    t = t_start + dt * np.arange(qd.size)
    m = t >= t_fit
    tau = t[m] - t_fit
    y = qd[m] - qd[0]

    def f(tt, a, b, c, ph):
        return a * np.exp(-b * tt) * np.sin(c * tt + ph)

    a0 = float(np.max(np.abs(y))) if y.size else 1.0
    best = None
    for ph0 in (0.0, np.pi / 2, np.pi, -np.pi / 2):
        try:
            popt, _ = curve_fit(f, tau, y, p0=[a0, b0, w0, ph0], maxfev=20000)
        except Exception:
            continue
        res = float(np.sum((f(tau, *popt) - y) ** 2))
        if best is None or res < best[0]:
            best = (res, popt)
    if best is None:
        return np.array([np.nan] * 4)
    a, b, c, ph = best[1]
    # one curve, several parameter sets: report a >= 0, c >= 0, phi in [0, 2 pi)
    if c < 0:
        c, ph = -c, np.pi - ph
    if a < 0:
        a, ph = -a, ph + np.pi
    return np.array([a, b, c, np.mod(ph, 2 * np.pi)])


def drude_admittance(omega, C, eta, nu):
    """Dipole term of the Drude admittance (Sec. 4), w in units of w_pe:
    Y_D = C (1/(i w) + (i w + nu)/eta^2)^{-1}."""
    omega = np.asarray(omega, dtype=np.float64)
    return C / (1.0 / (1j * omega) + (1j * omega + nu) / eta ** 2)


def drude_fit(omega, Y, w_lo=0.0, w_hi=1.0):
    """Least squares of int_{w_lo}^{w_hi} |Y_D(C, eta, nu; w) - Y(w)|^2 dw (Sec. 4:
    the integral I, here of the squared modulus, trapezoid rule on the given
    points) over C, eta > 0, nu > 0. Starting point: eta at the largest Re Y,
    nu its full width at half maximum. Returns (C, eta, nu, relative residual)."""
    from scipy.optimize import least_squares
    omega = np.asarray(omega, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.complex128)
    m = (omega >= w_lo) & (omega <= w_hi)
    w, y = omega[m], Y[m]
    if w.size < 5:
        raise ValueError("fewer than 5 points in the window")
    h = np.diff(w)
    wt = np.zeros(w.size)
    wt[:-1] += 0.5 * h
    wt[1:] += 0.5 * h
    sw = np.sqrt(wt)
    eta0, nu0 = peak_and_fwhm(w, y.real)
    if not nu0 > 0:
        nu0 = 0.1 * eta0
    g0 = drude_admittance(w, 1.0, eta0, nu0)
    C0 = float(np.sum(wt * (g0.conj() * y).real) / np.sum(wt * np.abs(g0) ** 2))

    def res(p):
        d = sw * (drude_admittance(w, p[0], p[1], p[2]) - y)
        return np.concatenate([d.real, d.imag])

    sol = least_squares(res, [C0, eta0, nu0], bounds=([-np.inf, 1e-12, 1e-12], [np.inf, np.inf, np.inf]),
                        xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    C, eta, nu = sol.x
    rel = float(np.sqrt(np.sum(res(sol.x) ** 2) / np.sum(wt * np.abs(y) ** 2)))
    return float(C), float(eta), float(nu), rel


def debye_over_R(T_e_eV, n_e_m3, R_m):
    """lambda_D / R with lambda_D = sqrt(eps0 T_e / (n_e e)) (T_e in eV)."""
    return float(np.sqrt(EPS0 * T_e_eV / (n_e_m3 * E_CHARGE)) / R_m)


def drude_K(nu_eff_wpe, T_e_eV, R_m, n_e_m3):
    """K of the paper's diagnostic nu_eff = K lambda_D w_pe / R (Sec. 4)."""
    return float(nu_eff_wpe / debye_over_R(T_e_eV, n_e_m3, R_m))


def drude_Te(nu_eff_wpe, K, R_m, n_e_m3):
    """T_e (eV) from nu_eff (units of w_pe) and K, the inverse of drude_K."""
    lam = nu_eff_wpe * R_m / K
    return float(lam * lam * n_e_m3 * E_CHARGE / EPS0)

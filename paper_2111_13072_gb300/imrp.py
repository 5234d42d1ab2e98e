"""Thin ctypes binding of the C ABI in include/imrp.h (argument marshalling only).

Every step of the hot path runs in the CUDA kernels of ``libimrp.so``; this
module only converts numpy arrays to pointers and error codes to exceptions.
It raises ImportError-like ``RuntimeError`` when the library is missing: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libimrp.so")

# Entry points declared in include/imrp.h (checked by the tests).
EXPORTS = [
    "imrp_default_params", "imrp_create", "imrp_destroy", "imrp_last_error", "imrp_set_stream",
    "imrp_load_particles", "imrp_step", "imrp_step_async", "imrp_sync", "imrp_get_qdiff",
    "imrp_get_field", "imrp_get_particles", "imrp_spectrum", "imrp_get_info", "imrp_profile_steps",
    "imrp_field_noalloc", "imrp_autotune", "imrp_batch_create", "imrp_batch_step", "imrp_batch_sync",
    "imrp_batch_destroy", "imrp_batch_last_error", "imrp_batch_set_stream", "imrp_footprint",
    "imrp_load_particles_async", "imrp_copy_qdiff_async", "imrp_drude_fit", "imrp_drude_k",
    "imrp_drude_te", "imrp_admittance", "imrp_fit_damped_sine", "imrp_sheath_solve",
    "imrp_set_ion_profile", "imrp_checkpoint", "imrp_restore", "imrp_batch_failed",
    "imrp_get_surface_charge", "imrp_fp32_peak", "imrp_ready", "imrp_set_species", "imrp_batch_autotune",
]
STAGES = ["sort", "reorder", "moments", "scans", "field"]

ERRORS = {-1: "IMRP_E_INVAL", -2: "IMRP_E_NOMEM", -3: "IMRP_E_CUDA", -4: "IMRP_E_TIMEOUT",
          -5: "IMRP_E_NAN", -6: "IMRP_E_STATE"}


class Params(ctypes.Structure):
    _fields_ = [
        ("R_E_m", ctypes.c_double), ("R_D_m", ctypes.c_double), ("eps_D", ctypes.c_double),
        ("R_out_m", ctypes.c_double), ("n_e_m3", ctypes.c_double), ("T_e_eV", ctypes.c_double),
        ("N", ctypes.c_int64), ("l_max", ctypes.c_int32), ("m0_only", ctypes.c_int32),
        ("dt", ctypes.c_double), ("drive_kind", ctypes.c_int32), ("wall_rule", ctypes.c_int32),
        ("V_volts", ctypes.c_double), ("width_wpe", ctypes.c_double), ("t0_wpe", ctypes.c_double),
        ("self_image", ctypes.c_int32), ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64),
        ("q_s", ctypes.c_double), ("nu_coll", ctypes.c_double),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_double), ("r_out", ctypes.c_double), ("n_tilde", ctypes.c_double),
        ("n_ion", ctypes.c_double), ("v_hat", ctypes.c_double), ("lambda_D", ctypes.c_double),
        ("omega_pe", ctypes.c_double), ("n", ctypes.c_int64), ("step", ctypes.c_int64),
        ("l_max", ctypes.c_int32), ("precision", ctypes.c_int32),
    ]


class IMRPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libimrp.so and declares the signatures of every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libimrp.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, c_void_p = ctypes.POINTER, ctypes.c_void_p
    pd = P(ctypes.c_double)
    L.imrp_default_params.argtypes = [P(Params)]
    L.imrp_default_params.restype = None
    L.imrp_create.argtypes = [P(Params), P(c_void_p)]
    L.imrp_destroy.argtypes = [c_void_p]
    L.imrp_last_error.argtypes = [c_void_p]
    L.imrp_last_error.restype = ctypes.c_char_p
    L.imrp_set_stream.argtypes = [c_void_p, c_void_p]
    L.imrp_load_particles.argtypes = [c_void_p, pd, pd, ctypes.c_int64]
    L.imrp_step.argtypes = [c_void_p, ctypes.c_int64, pd, pd]
    L.imrp_step_async.argtypes = [c_void_p, ctypes.c_int64]
    L.imrp_sync.argtypes = [c_void_p]
    L.imrp_get_qdiff.argtypes = [c_void_p, ctypes.c_int64, ctypes.c_int64, pd, pd]
    L.imrp_load_particles_async.argtypes = [c_void_p, pd, pd, ctypes.c_int64]
    L.imrp_copy_qdiff_async.argtypes = [c_void_p, ctypes.c_int64, ctypes.c_int64, pd, pd]
    L.imrp_get_field.argtypes = [c_void_p, pd]
    L.imrp_get_particles.argtypes = [c_void_p, pd, pd]
    L.imrp_spectrum.argtypes = [c_void_p, ctypes.c_int64, ctypes.c_double, pd, pd, pd, pd, pd, pd]
    L.imrp_get_info.argtypes = [c_void_p, P(Info)]
    L.imrp_profile_steps.argtypes = [c_void_p, ctypes.c_int64, pd]
    L.imrp_autotune.argtypes = [c_void_p, P(ctypes.c_int), P(ctypes.c_int)]
    L.imrp_batch_create.argtypes = [P(c_void_p), ctypes.c_int, P(c_void_p)]
    L.imrp_batch_step.argtypes = [c_void_p, ctypes.c_int64]
    L.imrp_batch_sync.argtypes = [c_void_p]
    L.imrp_batch_destroy.argtypes = [c_void_p]
    L.imrp_batch_set_stream.argtypes = [c_void_p, c_void_p]
    L.imrp_footprint.argtypes = [P(Params), ctypes.c_int64, P(ctypes.c_size_t)]
    L.imrp_batch_last_error.argtypes = [c_void_p]
    L.imrp_batch_failed.argtypes = [c_void_p]
    L.imrp_batch_last_error.restype = ctypes.c_char_p
    L.imrp_field_noalloc.argtypes = [P(Params), c_void_p, ctypes.c_int64, ctypes.c_int64, c_void_p, c_void_p]
    L.imrp_admittance.argtypes = [pd, pd, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                  ctypes.c_double, pd, pd, pd]
    L.imrp_fit_damped_sine.argtypes = [pd, ctypes.c_int64] + [ctypes.c_double] * 5 + [pd]
    L.imrp_drude_fit.argtypes = [pd, pd, pd, ctypes.c_int64, ctypes.c_double, ctypes.c_double, pd]
    L.imrp_drude_k.argtypes = [ctypes.c_double] * 4 + [pd]
    L.imrp_drude_te.argtypes = [ctypes.c_double] * 4 + [pd]
    L.imrp_sheath_solve.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int64] + [pd] * 5
    L.imrp_set_ion_profile.argtypes = [c_void_p, pd, ctypes.c_int64, ctypes.c_double, ctypes.c_double]
    pu32 = P(ctypes.c_uint32)
    L.imrp_checkpoint.argtypes = [c_void_p, pd, pd, pu32, P(ctypes.c_int64)]
    L.imrp_restore.argtypes = [c_void_p, pd, pd, pu32, ctypes.c_int64, ctypes.c_int64]
    L.imrp_get_surface_charge.argtypes = [c_void_p, pd, P(ctypes.c_int64)]
    L.imrp_fp32_peak.argtypes = [pd, P(ctypes.c_int)]
    L.imrp_ready.argtypes = [c_void_p, P(ctypes.c_int)]
    L.imrp_batch_autotune.argtypes = [c_void_p]
    L.imrp_set_species.argtypes = [c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    for name in EXPORTS:
        if name not in ("imrp_default_params", "imrp_last_error", "imrp_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_params() -> Params:
    p = Params()
    load_library().imrp_default_params(ctypes.byref(p))
    return p


def params_from_workload(w, **overrides) -> Params:
    """Copies a paper_2111_13072_gb300.inputs.Workload into Params."""
    p = default_params()
    p.R_E_m, p.R_D_m, p.eps_D = w.R_E_m, w.R_D_m, w.eps_D
    p.R_out_m, p.n_e_m3, p.T_e_eV = w.R_out_m, w.n_e_m3, w.T_e_eV
    p.N, p.l_max, p.dt = w.N, w.l_max, w.dt
    p.drive_kind, p.wall_rule, p.V_volts, p.width_wpe = w.drive_kind, w.wall_rule, w.V_volts, w.width_wpe
    p.self_image, p.precision, p.seed, p.m0_only = w.self_image, w.precision, w.seed, w.m0_only
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def field_noalloc(params: Params, x_dev_ptr: int, n: int, step: int, E_dev_ptr: int,
                  stream_ptr: int | None = None) -> None:
    """imrp_field_noalloc on caller-owned device buffers (FP64 [n][3] each)."""
    rc = load_library().imrp_field_noalloc(ctypes.byref(params), ctypes.c_void_p(x_dev_ptr), n, step,
                                           ctypes.c_void_p(E_dev_ptr), ctypes.c_void_p(stream_ptr or 0))
    if rc != 0:
        raise IMRPError(rc, "imrp_field_noalloc failed")


def fp32_peak():
    """imrp_fp32_peak: (measured FP32 FMA TFLOP/s of the current device, SM count)."""
    t, n = ctypes.c_double(), ctypes.c_int()
    rc = load_library().imrp_fp32_peak(ctypes.byref(t), ctypes.byref(n))
    if rc != 0:
        raise IMRPError(rc, "fp32_peak failed")
    return t.value, n.value


def admittance(q, u, dt: float, first_kick: float, n_freq: int = 1000, w_max: float = 2.0):
    """imrp_admittance: (omega, reY, imY) of host series q (Q_diff) and u (u_asy)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    om, re, im = np.zeros(n_freq), np.zeros(n_freq), np.zeros(n_freq)
    rc = load_library().imrp_admittance(_ptr(q), _ptr(u), q.size, dt, first_kick, n_freq, w_max,
                                        _ptr(om), _ptr(re), _ptr(im))
    if rc != 0:
        raise IMRPError(rc, "imrp_admittance failed")
    return om, re, im


def fit_damped_sine(q, dt: float, t_fit: float, t_end: float, w0: float, b0: float):
    """imrp_fit_damped_sine: (a, b, c, phi) of a e^{-b tau} sin(c tau + phi)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(4)
    rc = load_library().imrp_fit_damped_sine(_ptr(q), q.size, dt, t_fit, t_end, w0, b0, _ptr(out))
    if rc != 0:
        raise IMRPError(rc, "imrp_fit_damped_sine failed")
    return out


def drude_fit(omega, reY, imY, w_lo: float = 0.0, w_hi: float = 1.0):
    """imrp_drude_fit: (C, eta, nu, relative residual) of the Drude dipole
    admittance fitted to Y = reY + i imY over w_lo <= omega <= w_hi (units of w_pe)."""
    w = np.ascontiguousarray(omega, dtype=np.float64)
    re = np.ascontiguousarray(reY, dtype=np.float64)
    im = np.ascontiguousarray(imY, dtype=np.float64)
    out = np.zeros(4)
    rc = load_library().imrp_drude_fit(_ptr(w), _ptr(re), _ptr(im), w.size, w_lo, w_hi, _ptr(out))
    if rc != 0:
        raise IMRPError(rc, "imrp_drude_fit failed")
    return tuple(float(v) for v in out)


def drude_k(nu_eff_wpe: float, T_e_eV: float, R_m: float, n_e_m3: float) -> float:
    """imrp_drude_k: K of nu_eff = K lambda_D w_pe / R."""
    out = np.zeros(1)
    rc = load_library().imrp_drude_k(nu_eff_wpe, T_e_eV, R_m, n_e_m3, _ptr(out))
    if rc != 0:
        raise IMRPError(rc, "imrp_drude_k failed")
    return float(out[0])


def drude_te(nu_eff_wpe: float, K: float, R_m: float, n_e_m3: float) -> float:
    """imrp_drude_te: T_e (eV) from nu_eff (units of w_pe) and K."""
    out = np.zeros(1)
    rc = load_library().imrp_drude_te(nu_eff_wpe, K, R_m, n_e_m3, _ptr(out))
    if rc != 0:
        raise IMRPError(rc, "imrp_drude_te failed")
    return float(out[0])


def sheath_solve(lam: float, mass_ratio: float, r_out: float, n_grid: int = 1025) -> dict:
    """imrp_sheath_solve: the floating equilibrium of App. D on the grid
    r_k = 1 + k (r_out - 1)/(n_grid - 1): rhat, psi_wall, dpsi_wall, q_s,
    residual, and the arrays r, psi, dpsi, q_ion, q_elec."""
    psi, dpsi, qi, qe = (np.zeros(n_grid) for _ in range(4))
    out = np.zeros(5)
    rc = load_library().imrp_sheath_solve(lam, mass_ratio, r_out, n_grid, _ptr(psi), _ptr(dpsi),
                                          _ptr(qi), _ptr(qe), _ptr(out))
    if rc != 0:
        raise IMRPError(rc, "imrp_sheath_solve failed")
    r = 1.0 + (r_out - 1.0) * np.arange(n_grid) / (n_grid - 1)
    return dict(rhat=out[0], psi_wall=out[1], dpsi_wall=out[2], q_s=out[3], residual=out[4], r=r,
                psi=psi, dpsi=dpsi, q_ion=qi, q_elec=qe)


def footprint(params: Params, n_steps: int) -> int:
    """Device bytes of a context for these parameters and n_steps recorded steps."""
    out = ctypes.c_size_t()
    rc = load_library().imrp_footprint(ctypes.byref(params), n_steps, ctypes.byref(out))
    if rc != 0:
        raise IMRPError(rc, "imrp_footprint failed")
    return out.value


class Batch:
    """Steps several loaded Sim instances together (one captured graph per step pair)."""

    def __init__(self, sims):
        self._lib = load_library()
        self.sims = list(sims)
        arr = (ctypes.c_void_p * len(self.sims))(*[s._h for s in self.sims])
        h = ctypes.c_void_p()
        rc = self._lib.imrp_batch_create(arr, len(self.sims), ctypes.byref(h))
        if rc != 0:
            raise IMRPError(rc, "imrp_batch_create failed")
        self._h = h

    def _check(self, rc):
        if rc != 0:
            raise IMRPError(rc, self._lib.imrp_batch_last_error(self._h).decode())

    def set_stream(self, stream_ptr: int | None):
        self._check(self._lib.imrp_batch_set_stream(self._h, ctypes.c_void_p(stream_ptr or 0)))

    def step(self, n: int):
        self._check(self._lib.imrp_batch_step(self._h, n))

    def sync(self):
        self._check(self._lib.imrp_batch_sync(self._h))

    def autotune(self):
        """imrp_batch_autotune: the fastest CTA size of each batched field launch."""
        self._check(self._lib.imrp_batch_autotune(self._h))

    def failed_index(self) -> int:
        """imrp_batch_failed: index of the sim whose error the last call raised, or -1."""
        return int(self._lib.imrp_batch_failed(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.imrp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Sim:
    """One plasma instance on the current CUDA device."""

    def __init__(self, params: Params):
        self._lib = load_library()
        h = ctypes.c_void_p()
        rc = self._lib.imrp_create(ctypes.byref(params), ctypes.byref(h))
        if rc != 0:
            raise IMRPError(rc, "imrp_create failed")
        self._h = h
        self.params = params

    def _check(self, rc):
        if rc != 0:
            raise IMRPError(rc, self._lib.imrp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.imrp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream_ptr: int | None):
        self._check(self._lib.imrp_set_stream(self._h, ctypes.c_void_p(stream_ptr or 0)))

    def load(self, x, v):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        assert x.shape == v.shape and x.ndim == 2 and x.shape[1] == 3
        self._check(self._lib.imrp_load_particles(self._h, _ptr(x), _ptr(v), x.shape[0]))

    def checkpoint(self):
        """imrp_checkpoint: (x, v, ids, step) of the run in its storage order."""
        n = self.info().n
        x = np.zeros((n, 3)); v = np.zeros((n, 3))
        ids = np.zeros(n, dtype=np.uint32)
        step = ctypes.c_int64()
        self._check(self._lib.imrp_checkpoint(self._h, _ptr(x), _ptr(v),
                                              ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                              ctypes.byref(step)))
        return x, v, ids, int(step.value)

    def restore(self, x, v, ids, step: int):
        """imrp_restore: continues a run from imrp_checkpoint's output."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        assert x.shape == v.shape and x.ndim == 2 and x.shape[1] == 3 and ids.shape == (x.shape[0],)
        self._check(self._lib.imrp_restore(self._h, _ptr(x), _ptr(v),
                                           ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                           x.shape[0], step))

    def set_ion_profile(self, q_ion, q_elec_total: float, q_s: float):
        """imrp_set_ion_profile: immobile ions of a radial profile (units e n_inf R^3);
        q_ion = None restores the uniform background."""
        if q_ion is None:
            self._check(self._lib.imrp_set_ion_profile(self._h, None, 0, 1.0, 0.0))
            return
        q = np.ascontiguousarray(q_ion, dtype=np.float64)
        self._check(self._lib.imrp_set_ion_profile(self._h, _ptr(q), q.size, q_elec_total, q_s))

    def load_ptr(self, x_ptr: int, v_ptr: int, n: int):
        """Loads from host pointers (e.g. pinned torch tensors)."""
        P = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.imrp_load_particles(self._h, ctypes.cast(x_ptr, P), ctypes.cast(v_ptr, P), n))

    def load_async_ptr(self, x_ptr: int, v_ptr: int, n: int):
        """Streamed load from host pointers (pinned): returns without waiting."""
        P = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.imrp_load_particles_async(self._h, ctypes.cast(x_ptr, P), ctypes.cast(v_ptr, P), n))

    def copy_qdiff_async(self, first: int, count: int, q_ptr: int, u_ptr: int = 0):
        """Queues the copy of recorded Q_diff (and u_asy) samples to the given pointers."""
        P = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.imrp_copy_qdiff_async(self._h, first, count, ctypes.cast(q_ptr, P),
                                                      ctypes.cast(u_ptr, P)))

    def step(self, n: int, record: bool = True):
        q = np.zeros(n) if record else None
        u = np.zeros(n) if record else None
        self._check(self._lib.imrp_step(self._h, n, _ptr(q), _ptr(u)))
        return q, u

    def step_ptr(self, n: int, q_ptr: int):
        P = ctypes.POINTER(ctypes.c_double)
        self._check(self._lib.imrp_step(self._h, n, ctypes.cast(q_ptr, P), None))

    def step_async(self, n: int):
        self._check(self._lib.imrp_step_async(self._h, n))

    def sync(self):
        self._check(self._lib.imrp_sync(self._h))

    def qdiff(self, first=0, count=None):
        info = self.info()
        count = info.step - first if count is None else count
        q, u = np.zeros(count), np.zeros(count)
        self._check(self._lib.imrp_get_qdiff(self._h, first, count, _ptr(q), _ptr(u)))
        return q, u

    def field(self):
        n = self.info().n
        E = np.zeros((n, 3))
        self._check(self._lib.imrp_get_field(self._h, _ptr(E)))
        return E

    def particles(self):
        n = self.info().n
        x, v = np.zeros((n, 3)), np.zeros((n, 3))
        self._check(self._lib.imrp_get_particles(self._h, _ptr(x), _ptr(v)))
        return x, v

    def set_species(self, n_electrons: int, ion_charge: float, ion_mass: float, background_ions: float = 0.0):
        """imrp_set_species: particles with id >= n_electrons are mobile ions."""
        self._check(self._lib.imrp_set_species(self._h, int(n_electrons), float(ion_charge), float(ion_mass),
                                               float(background_ions)))

    def ready(self) -> bool:
        """imrp_ready: True when the context's queued work has finished (no wait)."""
        r = ctypes.c_int()
        self._check(self._lib.imrp_ready(self._h, ctypes.byref(r)))
        return bool(r.value)

    def surface_charge(self):
        """imrp_get_surface_charge: (Q_S in super-particle charges, probe absorptions)."""
        q, k = ctypes.c_double(), ctypes.c_int64()
        self._check(self._lib.imrp_get_surface_charge(self._h, ctypes.byref(q), ctypes.byref(k)))
        return q.value, k.value

    def spectrum(self, n_freq: int = 1000, w_max: float = 2.0, fit: bool = True):
        om, re, im = np.zeros(n_freq), np.zeros(n_freq), np.zeros(n_freq)
        wr, dw = ctypes.c_double(), ctypes.c_double()
        f = np.zeros(4)
        self._check(self._lib.imrp_spectrum(self._h, n_freq, w_max, _ptr(om), _ptr(re), _ptr(im),
                                            ctypes.pointer(wr), ctypes.pointer(dw),
                                            _ptr(f) if fit else None))
        return {"omega": om, "reY": re, "imY": im, "w_res": wr.value, "dw": dw.value,
                "fit": f if fit else None}

    def profile_steps(self, n: int) -> dict:
        """Takes n real steps with per-stage CUDA events; returns summed ms per stage."""
        ms = np.zeros(len(STAGES))
        self._check(self._lib.imrp_profile_steps(self._h, n, _ptr(ms)))
        return dict(zip(STAGES, ms.tolist()))

    def autotune(self):
        """Picks the field CTA size and the group-scan segment length by timing; returns (wpb, gseg)."""
        w, c = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.imrp_autotune(self._h, ctypes.byref(w), ctypes.byref(c)))
        return w.value, c.value

    def info(self) -> Info:
        i = Info()
        self._check(self._lib.imrp_get_info(self._h, ctypes.byref(i)))
        return i

"""ctypes binding of libpertgb (include/pertgb.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name.  Arrays may be
torch tensors (CUDA or CPU) or NumPy arrays; their data pointers are passed
through unchanged, and the library decides whether a pointer is host or
device memory.  Nothing here computes any part of the method, and there is
no fallback: if the shared library or a CUDA device is missing, the calls
raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpertgb.so")

PGB_OK, PGB_EINVAL, PGB_ESTATE, PGB_ENOMEM, PGB_ECUDA, PGB_ETIMEOUT = 0, -1, -2, -3, -4, -5
PGB_FP64, PGB_FP32, PGB_TC_TF32X3, PGB_TC_BF16X3 = 0, 1, 2, 3
PGB_G2_FULL, PGB_G_ABS = 0, 1
PRECISIONS = {"fp64": PGB_FP64, "fp32": PGB_FP32, "tf32x3": PGB_TC_TF32X3, "bf16x3": PGB_TC_BF16X3}

DIAG_SYMBOLS = ("pgb_diag_bands", "pgb_selftest_heevj", "pgb_selftest_heevj_device", "pgb_selftest_wait_timeout",
                "pgb_diag_alloc_count", "pgb_diag_fail_alloc", "pgb_diag_delta_weights",
                "pgb_diag_fp64_rate", "pgb_diag_bands_mixed", "pgb_diag_phonons_mixed")
ABI_SYMBOLS = (
    "pgb_create", "pgb_destroy", "pgb_last_error", "pgb_status_string", "pgb_set_model",
    "pgb_set_grids", "pgb_get_grid_energies", "pgb_window", "pgb_interpolate_g",
    "pgb_scattering_rates", "pgb_build_collision", "pgb_collision_energies", "pgb_collision",
    "pgb_step_rk4", "pgb_launch_count", "pgb_profile", "pgb_profile_read",
    "pgb_scattering_rates_noalloc", "pgb_build_collision_grid", "pgb_collision_list",
    "pgb_collision_set_g2", "pgb_collision_vjp", "pgb_rk4_adjoint",
    "pgb_set_lattice", "pgb_set_polar", "pgb_long_range_g", "pgb_band_velocities", "pgb_transport",
    "pgb_scattering_rates_mc", "pgb_population",
    "pgb_batch_create", "pgb_batch_rates", "pgb_batch_tuning", "pgb_batch_set_precision", "pgb_batch_last_error",
    "pgb_batch_destroy",
)
PGB_Q_UNIFORM, PGB_Q_CAUCHY = 0, 1
PGB_NOALLOC_SCRATCH_BYTES = 64 << 20
PROF_QSUM, PROF_RSUM, PROF_EPILOGUE, PROF_COLLISION, PROF_BANDS, PROF_ADJOINT = 0, 1, 2, 3, 4, 5


class PgbModel(C.Structure):
    _fields_ = [
        ("nw", C.c_int), ("nat", C.c_int), ("mass", C.c_void_p),
        ("nR_H", C.c_int), ("R_H", C.c_void_p), ("H", C.c_void_p),
        ("nR_D", C.c_int), ("R_D", C.c_void_p), ("D", C.c_void_p),
        ("nR_ge", C.c_int), ("R_ge", C.c_void_p), ("nR_gp", C.c_int), ("R_gp", C.c_void_p),
        ("g", C.c_void_p), ("g_is_double", C.c_int),
    ]


class PgbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pertgb status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libpertgb.so (build it with ``paper_2002_02045_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run `python -m paper_2002_02045_gb300.build` first")
    lib = C.CDLL(path)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "pgb_create": (I, [C.POINTER(P), I, P]),
        "pgb_destroy": (None, [P]),
        "pgb_last_error": (C.c_char_p, [P]),
        "pgb_status_string": (C.c_char_p, [I]),
        "pgb_set_model": (I, [P, C.POINTER(PgbModel)]),
        "pgb_set_grids": (I, [P, P, P]),
        "pgb_get_grid_energies": (I, [P, P, P]),
        "pgb_window": (I, [P, D, D, P, C.POINTER(I64)]),
        "pgb_interpolate_g": (I, [P, P, I64, P, I64, I, I, P]),
        "pgb_scattering_rates": (I, [P, P, I64, D, D, D, I, P, P]),
        "pgb_build_collision": (I, [P, I, I, D, D, I64, P, P, P, P]),
        "pgb_collision_energies": (I, [P, P, C.POINTER(I64)]),
        "pgb_build_collision_grid": (I, [P, I, I, D, D, D, D, C.POINTER(I64)]),
        "pgb_collision_list": (I, [P, P, P, P, P]),
        "pgb_collision": (I, [P, P, P]),
        "pgb_step_rk4": (I, [P, P, D, I64]),
        "pgb_collision_set_g2": (I, [P, P]),
        "pgb_collision_vjp": (I, [P, P, P, P, P]),
        "pgb_rk4_adjoint": (I, [P, P, D, I64, I64, P, P, P, P]),
        "pgb_set_lattice": (I, [P, P, P]),
        "pgb_set_polar": (I, [P, P, P, D]),
        "pgb_long_range_g": (I, [P, P, I64, P]),
        "pgb_band_velocities": (I, [P, P, I64, P]),
        "pgb_transport": (I, [P, D, I, I, D, P, P, C.POINTER(I64), P, P]),
        "pgb_scattering_rates_mc": (I, [P, P, I64, P, I64, I, D, D, D, D, I, P, P]),
        "pgb_population": (I, [P, P, P, I64, P]),
        "pgb_batch_create": (I, [C.POINTER(P), P, I]),
        "pgb_batch_rates": (I, [P, P, P, D, P, D, P]),
        "pgb_batch_tuning": (I, [P, C.POINTER(I), C.POINTER(I), P, C.POINTER(I64)]),
        "pgb_batch_set_precision": (I, [P, I]),
        "pgb_batch_last_error": (C.c_char_p, [P]),
        "pgb_batch_destroy": (None, [P]),
        "pgb_launch_count": (I64, [P]),
        "pgb_profile": (I, [P, I]),
        "pgb_scattering_rates_noalloc": (I, [P, P, I64, D, D, D, P]),
        "pgb_profile_read": (I, [P, I, C.POINTER(D), C.POINTER(I64)]),
        "pgb_diag_bands": (I, [P, P, I64, P, P, P]),
        "pgb_diag_bands_mixed": (I, [P, P, I64, P, P, P]),
        "pgb_diag_phonons_mixed": (I, [P, P, I64, P, P, P]),
        "pgb_selftest_heevj": (I, [I, I, P, P, P]),
        "pgb_selftest_heevj_device": (I, [P, I, I, P, P, P]),
        "pgb_selftest_wait_timeout": (I, [P, C.c_longlong]),
        "pgb_diag_alloc_count": (I64, []),
        "pgb_diag_fail_alloc": (None, [I64]),
        "pgb_diag_delta_weights": (I, [P, I64, P, P, P, D, D, P]),
        "pgb_diag_fp64_rate": (I, [P, C.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Data pointer of a torch tensor or NumPy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("arrays passed to pertgb must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to pertgb must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _check_dtype(x, kind):
    if x is None:
        return
    name = str(getattr(x, "dtype", ""))
    if kind not in name:
        raise TypeError(f"expected a {kind} array, got {name}")


class Context:
    """One pgb_ctx on one CUDA device and stream (the current torch stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        self._h = C.c_void_p()
        st = self.lib.pgb_create(C.byref(self._h), device, C.c_void_p(stream))
        if st != PGB_OK:
            raise PgbError(st, "pgb_create failed (no usable CUDA device?)")
        self._keep = []

    def close(self):
        if self._h:
            self.lib.pgb_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != PGB_OK:
            raise PgbError(st, self.lib.pgb_last_error(self._h).decode())

    # -- ABI ---------------------------------------------------------------
    def pgb_set_model(self, model):
        g = np.ascontiguousarray(model.g)
        if g.dtype == np.complex64:
            gd = 0
        elif g.dtype == np.complex128:
            gd = 1
        else:
            raise TypeError("g must be complex64 or complex128")
        arrs = dict(
            mass=np.ascontiguousarray(model.mass, np.float64),
            R_H=np.ascontiguousarray(model.R_H, np.int32), H=np.ascontiguousarray(model.H, np.complex128),
            R_D=np.ascontiguousarray(model.R_D, np.int32), D=np.ascontiguousarray(model.D, np.float64),
            R_ge=np.ascontiguousarray(model.R_ge, np.int32), R_gp=np.ascontiguousarray(model.R_gp, np.int32),
            g=g)
        m = PgbModel(nw=model.H.shape[1], nat=len(model.mass), mass=_ptr(arrs["mass"]),
                     nR_H=len(model.R_H), R_H=_ptr(arrs["R_H"]), H=_ptr(arrs["H"]),
                     nR_D=len(model.R_D), R_D=_ptr(arrs["R_D"]), D=_ptr(arrs["D"]),
                     nR_ge=len(model.R_ge), R_ge=_ptr(arrs["R_ge"]), nR_gp=len(model.R_gp),
                     R_gp=_ptr(arrs["R_gp"]), g=_ptr(g), g_is_double=gd)
        self._chk(self.lib.pgb_set_model(self._h, C.byref(m)))
        self.nw = int(model.H.shape[1])
        self.nmode = 3 * len(model.mass)

    def pgb_set_lattice(self, lattice, tau):
        lat = np.ascontiguousarray(lattice, np.float64).reshape(9)
        t = np.ascontiguousarray(tau, np.float64).reshape(-1)
        self._chk(self.lib.pgb_set_lattice(self._h, _ptr(lat), _ptr(t)))

    def pgb_set_polar(self, zstar, eps_inf=None, ewald_lambda=0.0):
        if zstar is None:
            self._chk(self.lib.pgb_set_polar(self._h, None, None, 0.0))
            return
        z = np.ascontiguousarray(zstar, np.float64).reshape(-1)
        e = np.ascontiguousarray(eps_inf, np.float64).reshape(9)
        self._chk(self.lib.pgb_set_polar(self._h, _ptr(z), _ptr(e), float(ewald_lambda)))

    def pgb_long_range_g(self, qpts, out):
        _check_dtype(qpts, "float64")
        _check_dtype(out, "float64")
        self._chk(self.lib.pgb_long_range_g(self._h, _ptr(qpts), len(qpts), _ptr(out)))

    def pgb_band_velocities(self, k_idx, v_out):
        _check_dtype(k_idx, "int32")
        _check_dtype(v_out, "float64")
        self._chk(self.lib.pgb_band_velocities(self._h, _ptr(k_idx), len(k_idx), _ptr(v_out)))

    def pgb_transport(self, mu, precision, max_iter, tol, F_out=None, tau_out=None):
        """Returns (mobility_rta [3,3], mobility [3,3], iterations) in cm^2/(V s)."""
        _check_dtype(F_out, "float64")
        _check_dtype(tau_out, "float64")
        mr = np.zeros(9)
        mi = np.zeros(9)
        it = C.c_int64(0)
        self._chk(self.lib.pgb_transport(self._h, float(mu), int(precision), int(max_iter), float(tol), _ptr(mr),
                                         _ptr(mi), C.byref(it), _ptr(F_out), _ptr(tau_out)))
        return mr.reshape(3, 3), mi.reshape(3, 3), int(it.value)

    def pgb_scattering_rates_mc(self, kpts, u, sampling, width, T, mu, sigma, precision, gamma_out,
                                stderr_out=None):
        for a in (kpts, u, gamma_out, stderr_out):
            _check_dtype(a, "float64")
        self._chk(self.lib.pgb_scattering_rates_mc(self._h, _ptr(kpts), len(kpts), _ptr(u), len(u), int(sampling),
                                                   float(width), float(T), float(mu), float(sigma), int(precision),
                                                   _ptr(gamma_out), _ptr(stderr_out)))

    def pgb_population(self, f, E, N_out):
        for a in (f, E, N_out):
            _check_dtype(a, "float64")
        self._chk(self.lib.pgb_population(self._h, _ptr(f), _ptr(E), len(E), _ptr(N_out)))

    def pgb_set_grids(self, kgrid, qgrid):
        kg = (C.c_int * 3)(*kgrid)
        qg = (C.c_int * 3)(*qgrid)
        self._chk(self.lib.pgb_set_grids(self._h, kg, qg))
        self.kgrid, self.qgrid = tuple(kgrid), tuple(qgrid)

    def pgb_get_grid_energies(self, eps, hw):
        _check_dtype(eps, "float64")
        _check_dtype(hw, "float64")
        self._chk(self.lib.pgb_get_grid_energies(self._h, _ptr(eps), _ptr(hw)))

    def pgb_window(self, e_lo, e_hi, k_idx_out):
        _check_dtype(k_idx_out, "int32")
        n = C.c_int64(0)
        self._chk(self.lib.pgb_window(self._h, float(e_lo), float(e_hi), _ptr(k_idx_out), C.byref(n)))
        return int(n.value)

    def pgb_interpolate_g(self, kpts, qpts, precision, out_mode, out):
        _check_dtype(kpts, "float64")
        _check_dtype(qpts, "float64")
        _check_dtype(out, "float64")
        self._chk(self.lib.pgb_interpolate_g(self._h, _ptr(kpts), len(kpts), _ptr(qpts), len(qpts),
                                             int(precision), int(out_mode), _ptr(out)))

    def pgb_scattering_rates(self, k_idx, T, mu, sigma, precision, gamma_out, gamma_mode_out=None):
        _check_dtype(k_idx, "int32")
        _check_dtype(gamma_out, "float64")
        _check_dtype(gamma_mode_out, "float64")
        self._chk(self.lib.pgb_scattering_rates(self._h, _ptr(k_idx), len(k_idx), float(T), float(mu),
                                                float(sigma), int(precision), _ptr(gamma_out),
                                                _ptr(gamma_mode_out)))

    def pgb_scattering_rates_noalloc(self, k_idx, T, mu, sigma, gamma_out):
        _check_dtype(k_idx, "int32")
        _check_dtype(gamma_out, "float64")
        self._chk(self.lib.pgb_scattering_rates_noalloc(self._h, _ptr(k_idx), len(k_idx), float(T), float(mu),
                                                        float(sigma), _ptr(gamma_out)))

    def pgb_build_collision(self, band_lo, band_hi, T, sigma, row, col, mode, g2):
        for a, k in ((row, "int32"), (col, "int32"), (mode, "int32"), (g2, "float32")):
            _check_dtype(a, k)
        n = len(row)
        if not (len(col) == len(mode) == len(g2) == n):
            raise ValueError("row, col, mode, g2 must have equal length")
        self._chk(self.lib.pgb_build_collision(self._h, int(band_lo), int(band_hi), float(T), float(sigma),
                                               n, _ptr(row), _ptr(col), _ptr(mode), _ptr(g2)))

    def pgb_build_collision_grid(self, band_lo, band_hi, e_lo, e_hi, T, sigma):
        n = C.c_int64(0)
        self._chk(self.lib.pgb_build_collision_grid(self._h, int(band_lo), int(band_hi), float(e_lo), float(e_hi),
                                                    float(T), float(sigma), C.byref(n)))
        return int(n.value)

    def pgb_collision_list(self, row=None, col=None, mode=None, g2=None):
        for a, k in ((row, "int32"), (col, "int32"), (mode, "int32"), (g2, "float32")):
            _check_dtype(a, k)
        self._chk(self.lib.pgb_collision_list(self._h, _ptr(row), _ptr(col), _ptr(mode), _ptr(g2)))

    def pgb_collision_energies(self, eps_state=None):
        n = C.c_int64(0)
        _check_dtype(eps_state, "float64")
        self._chk(self.lib.pgb_collision_energies(self._h, _ptr(eps_state), C.byref(n)))
        return int(n.value)

    def pgb_collision(self, f, I_out):
        _check_dtype(f, "float64")
        _check_dtype(I_out, "float64")
        self._chk(self.lib.pgb_collision(self._h, _ptr(f), _ptr(I_out)))

    def pgb_step_rk4(self, f, dt_fs, nsteps):
        _check_dtype(f, "float64")
        self._chk(self.lib.pgb_step_rk4(self._h, _ptr(f), float(dt_fs), int(nsteps)))

    def pgb_collision_set_g2(self, g2):
        _check_dtype(g2, "float32")
        self._chk(self.lib.pgb_collision_set_g2(self._h, _ptr(g2)))

    def pgb_collision_vjp(self, f, lam, vjp_f, vjp_g2=None):
        for a in (f, lam, vjp_f, vjp_g2):
            _check_dtype(a, "float64")
        self._chk(self.lib.pgb_collision_vjp(self._h, _ptr(f), _ptr(lam), _ptr(vjp_f), _ptr(vjp_g2)))

    def pgb_rk4_adjoint(self, f0, dt_fs, nsteps, checkpoint, lam_end, lam_0, dL_dg2=None, f_end=None):
        for a in (f0, lam_end, lam_0, dL_dg2, f_end):
            _check_dtype(a, "float64")
        self._chk(self.lib.pgb_rk4_adjoint(self._h, _ptr(f0), float(dt_fs), int(nsteps), int(checkpoint),
                                           _ptr(lam_end), _ptr(lam_0), _ptr(dL_dg2), _ptr(f_end)))

    def pgb_launch_count(self):
        return int(self.lib.pgb_launch_count(self._h))

    def pgb_diag_bands(self, pts, Hk=None, eps=None, U=None):
        self._chk(self.lib.pgb_diag_bands(self._h, _ptr(pts), len(pts), _ptr(Hk), _ptr(eps), _ptr(U)))

    def pgb_diag_bands_mixed(self, pts, Hp=None, eps=None, U=None):
        self._chk(self.lib.pgb_diag_bands_mixed(self._h, _ptr(pts), len(pts), _ptr(Hp), _ptr(eps), _ptr(U)))

    def pgb_diag_phonons_mixed(self, pts, Dp=None, w2=None, e=None):
        self._chk(self.lib.pgb_diag_phonons_mixed(self._h, _ptr(pts), len(pts), _ptr(Dp), _ptr(w2), _ptr(e)))

    def pgb_diag_delta_weights(self, en, em, hw, eps_ref, sigma, out):
        for a in (en, em, hw):
            _check_dtype(a, "float64")
        _check_dtype(out, "float32")
        self._chk(self.lib.pgb_diag_delta_weights(self._h, len(en), _ptr(en), _ptr(em), _ptr(hw), float(eps_ref),
                                                  float(sigma), _ptr(out)))

    def pgb_diag_fp64_rate(self):
        t = C.c_double(0.0)
        self._chk(self.lib.pgb_diag_fp64_rate(self._h, C.byref(t)))
        return float(t.value)

    def pgb_profile(self, enable):
        self._chk(self.lib.pgb_profile(self._h, 1 if enable else 0))

    def pgb_profile_read(self, kernel_class):
        ms = C.c_double(0.0)
        n = C.c_int64(0)
        self._chk(self.lib.pgb_profile_read(self._h, int(kernel_class), C.byref(ms), C.byref(n)))
        return float(ms.value), int(n.value)


class Batch:
    """pgb_batch over several Contexts (same device); rates of every instance in one graph launch."""

    def __init__(self, contexts):
        self.lib = load()
        self._ctx = list(contexts)          # keep the contexts alive
        arr = (C.c_void_p * len(self._ctx))(*[c._h.value for c in self._ctx])
        self._h = C.c_void_p()
        st = self.lib.pgb_batch_create(C.byref(self._h), arr, len(self._ctx))
        if st != PGB_OK:
            raise PgbError(st, "pgb_batch_create failed: " + " / ".join(
                c.lib.pgb_last_error(c._h).decode() for c in self._ctx))

    def close(self):
        if self._h:
            self.lib.pgb_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pgb_batch_rates(self, k_lists, T, mus, sigma, outs):
        n = len(self._ctx)
        keep = [np.ascontiguousarray(k, np.int32) if isinstance(k, (list, tuple)) else k for k in k_lists]
        kp = (C.c_void_p * n)(*[_ptr(k) for k in keep])
        nk = (C.c_int64 * n)(*[len(k) for k in keep])
        mu = (C.c_double * n)(*[float(m) for m in mus])
        op = (C.c_void_p * n)(*[_ptr(o) for o in outs])
        st = self.lib.pgb_batch_rates(self._h, kp, nk, float(T), mu, float(sigma), op)
        if st != PGB_OK:
            raise PgbError(st, self.lib.pgb_batch_last_error(self._h).decode())

    def pgb_batch_set_precision(self, precision):
        st = self.lib.pgb_batch_set_precision(self._h, int(precision))
        if st != 0:
            raise PgbError(st, self.lib.pgb_batch_last_error(self._h).decode())

    def pgb_batch_tuning(self):
        qt, nt, gl = C.c_int(0), C.c_int(0), C.c_int64(0)
        ms = (C.c_float * 4)()
        self.lib.pgb_batch_tuning(self._h, C.byref(qt), C.byref(nt), ms, C.byref(gl))
        return {"tile_q": qt.value, "threads": nt.value, "candidate_ms": list(ms), "graph_launches": gl.value}

"""Thin ctypes binding of libmdbs.so (include/mdbs.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels.  Loading fails loudly
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdbs.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_DIVERGED, ERR_NOT_CONVERGED = 0, -1, -2, -3, -4, -5


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("h", C.c_double)]


class Fluids(C.Structure):
    _fields_ = [("rho_l", C.c_double), ("mu_l", C.c_double), ("rho_g", C.c_double), ("mu_g", C.c_double),
                ("sigma", C.c_double), ("g", C.c_double * 3)]


class Closures(C.Structure):
    _fields_ = [("kr_model", C.c_int32), ("pc_model", C.c_int32), ("kr_m", C.c_double),
                ("a_l_irr", C.c_double), ("a_g_irr", C.c_double), ("pc0", C.c_double),
                ("pc_beta", C.c_double), ("pc_m", C.c_double), ("a_pc_irr", C.c_double),
                ("a_pc_max", C.c_double), ("pc_eps", C.c_double), ("porous_density", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("dt", C.c_double), ("cfl", C.c_double), ("dt_max", C.c_double), ("c_alpha", C.c_double),
                ("p_tol", C.c_double), ("n_corr", C.c_int32), ("mom_sweeps", C.c_int32),
                ("max_cg", C.c_int32), ("mg_nu1", C.c_int32), ("mg_nu2", C.c_int32),
                ("mg_coarse_sweeps", C.c_int32), ("precision", C.c_int32), ("bc", C.c_int32 * 6),
                ("inlet_u", C.c_double), ("inlet_alpha", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("time", C.c_double), ("dt", C.c_double),
                ("cg_iters", C.c_int32 * 8), ("cg_resid", C.c_double * 8), ("cg_iters_total", C.c_int64),
                ("not_converged", C.c_int32), ("mass", C.c_double), ("boundary_in", C.c_double),
                ("alpha_min", C.c_double), ("alpha_max", C.c_double), ("kernel_launches", C.c_int64)]


_D = C.POINTER(C.c_double)
_lib = None
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)
_hook = None  # keeps the ctypes callbacks of the installed allocator alive


class Tuning(C.Structure):
    """Schedule of the multigrid kernels (mdbs_tuning); results do not depend on it."""
    _fields_ = [("smooth_rows", C.c_int32), ("tail_cells", C.c_int32), ("snake", C.c_int32),
                ("sweep_kz", C.c_int32), ("tail_ctas", C.c_int32), ("coarse_coop", C.c_int32),
                ("vec_sweeps", C.c_int32)]

    def as_dict(self):
        return {"smooth_rows": self.smooth_rows, "tail_cells": self.tail_cells, "snake": self.snake,
                "sweep_kz": self.sweep_kz, "tail_ctas": self.tail_ctas, "coarse_coop": self.coarse_coop,
                "vec_sweeps": self.vec_sweeps}


def _tuning(t):
    if isinstance(t, Tuning):
        return t
    return Tuning(t["smooth_rows"], t["tail_cells"], t["snake"], t["sweep_kz"], t.get("tail_ctas", 1),
                  t.get("coarse_coop", 0), t.get("vec_sweeps", 0))


class MdbsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("mdbs error %d: %s" % (code, msg))
        self.code = code


def lib():
    """Loads libmdbs.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmdbs.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        L.mdbs_create.argtypes = [C.POINTER(Grid), _D, _D, C.POINTER(Fluids), C.c_double, C.POINTER(Closures),
                                  C.POINTER(Options), C.POINTER(C.c_void_p)]
        L.mdbs_set_fields.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        L.mdbs_step.argtypes = [C.c_void_p, C.c_int32]
        L.mdbs_get_fields.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        L.mdbs_destroy.argtypes = [C.c_void_p]
        L.mdbs_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.mdbs_last_error.argtypes = [C.c_void_p]
        L.mdbs_last_error.restype = C.c_char_p
        L.mdbs_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.mdbs_bytes_required.argtypes = [C.POINTER(Grid), C.c_int32]
        L.mdbs_bytes_required.restype = C.c_size_t
        L.mdbs_profile_enable.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
        L.mdbs_profile_count.restype = C.c_int32
        L.mdbs_profile_read.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_char_p), _D,
                                        C.POINTER(C.c_int64)]
        L.mdbs_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]
        L.mdbs_batch_step.argtypes = [C.c_void_p, C.c_int32]
        L.mdbs_batch_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.mdbs_batch_last_error.argtypes = [C.c_void_p]
        L.mdbs_batch_last_error.restype = C.c_char_p
        L.mdbs_batch_destroy.argtypes = [C.c_void_p]
        L.mdbs_batch_add.argtypes = [C.c_void_p, C.c_void_p]
        L.mdbs_batch_remove.argtypes = [C.c_void_p, C.c_void_p]
        L.mdbs_set_allocator.argtypes = [ALLOC_FN, FREE_FN, C.c_void_p]
        L.mdbs_field_stats_static.argtypes = [C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p, C.c_void_p]
        L.mdbs_debug_array.argtypes = [C.c_void_p, C.c_char_p, _D, C.c_int64]
        L.mdbs_debug_array.restype = C.c_int64
        L.mdbs_check_bounded_wait.argtypes = [_D]
        for nm in ("mdbs_set_tuning", "mdbs_get_tuning", "mdbs_batch_set_tuning", "mdbs_batch_get_tuning"):
            getattr(L, nm).argtypes = [C.c_void_p, C.POINTER(Tuning)]
        for nm in ("mdbs_autotune", "mdbs_batch_autotune"):
            getattr(L, nm).argtypes = [C.c_void_p, C.c_int32, C.POINTER(Tuning), _D, C.c_int32,
                                       C.POINTER(C.c_int32)]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def structs_from_case(case):
    grid = Grid(case.nx, case.ny, case.nz, case.h)
    fl = Fluids(case.rho_l, case.mu_l, case.rho_g, case.mu_g, case.sigma, (C.c_double * 3)(*case.g))
    cl = Closures(case.kr_model, case.pc_model, case.kr_m, case.a_l_irr, case.a_g_irr, case.pc0, case.pc_beta,
                  case.pc_m, case.a_pc_irr, case.a_pc_max, case.pc_eps, case.porous_density)
    op = Options(case.dt, case.cfl, case.dt_max, case.c_alpha, case.p_tol, case.n_corr, case.mom_sweeps,
                 case.max_cg, case.mg_nu1, case.mg_nu2, case.mg_coarse_sweeps, case.precision,
                 (C.c_int32 * 6)(*case.bc), case.inlet_u, case.inlet_alpha)
    return grid, fl, cl, op


def field_stats_static(cells, cell_volume, porosity_ptr, alpha_ptr, p_ptr, out_ptr, stream=0):
    """mdbs_field_stats_static on caller-owned device buffers (integer device addresses);
    allocates nothing.  out receives volume, alpha min, alpha max, non-finite count."""
    rc = lib().mdbs_field_stats_static(int(cells), float(cell_volume), C.c_void_p(porosity_ptr),
                                       C.c_void_p(alpha_ptr), C.c_void_p(p_ptr), C.c_void_p(out_ptr),
                                       C.c_void_p(stream))
    if rc != OK:
        raise MdbsError(rc, "mdbs_field_stats_static rejected the call")


def bytes_required(case, precision=None):
    g = Grid(case.nx, case.ny, case.nz, case.h)
    return int(lib().mdbs_bytes_required(C.byref(g), case.precision if precision is None else precision))


def check_bounded_wait():
    """Runs the bounded-wait self-test; returns the device-measured wait in seconds."""
    w = C.c_double()
    rc = lib().mdbs_check_bounded_wait(C.byref(w))
    if rc != OK:
        raise MdbsError(rc, lib().mdbs_last_error(None).decode())
    return w.value


def kernel_names():
    out = []
    for i in range(lib().mdbs_profile_count()):
        nm = C.c_char_p()
        lib().mdbs_profile_read(None, i, C.byref(nm), None, None)
        out.append(nm.value.decode() if nm.value else "")
    return out


class Simulation:
    """One device-resident simulation (mdbs_create ... mdbs_destroy)."""

    def __init__(self, case, set_fields=True):
        self.case = case
        self.n = (case.nx, case.ny, case.nz)
        grid, fl, cl, op = structs_from_case(case)
        phi, k = _f64(case.porosity.ravel()), _f64(case.permeability.ravel())
        h = C.c_void_p()
        rc = lib().mdbs_create(C.byref(grid), _ptr(phi), _ptr(k), C.byref(fl), case.theta_deg, C.byref(cl),
                               C.byref(op), C.byref(h))
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_last_error(None).decode())
        self.h = h
        if set_fields:
            self.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)

    def _check(self, rc):
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_last_error(self.h).decode())

    def set_fields(self, alpha, ux, uy, uz, p):
        a, x, y, pp = (_f64(v.ravel()) for v in (alpha, ux, uy, p))
        z = _f64(uz.ravel()) if uz is not None and self.n[2] > 1 else None
        self._check(lib().mdbs_set_fields(self.h, _ptr(a), _ptr(x), _ptr(y), _ptr(z), _ptr(pp)))

    def step(self, n=1):
        self._check(lib().mdbs_step(self.h, int(n)))

    def fields(self):
        nx, ny, nz = self.n
        out = {"alpha": np.zeros(nx * ny * nz), "p": np.zeros(nx * ny * nz),
               "ux": np.zeros((nx + 1) * ny * nz), "uy": np.zeros(nx * (ny + 1) * nz),
               "uz": np.zeros(nx * ny * (nz + 1)) if nz > 1 else np.zeros(0)}
        self._check(lib().mdbs_get_fields(self.h, _ptr(out["alpha"]), _ptr(out["ux"]), _ptr(out["uy"]),
                                          _ptr(out["uz"]) if nz > 1 else None, _ptr(out["p"])))
        return out

    def stats(self):
        st = Stats()
        self._check(lib().mdbs_get_stats(self.h, C.byref(st)))
        return {"steps": st.steps, "time": st.time, "dt": st.dt,
                "cg_iters": list(st.cg_iters)[: self.case.n_corr],
                "cg_resid": list(st.cg_resid)[: self.case.n_corr],
                "cg_iters_total": st.cg_iters_total, "not_converged": st.not_converged,
                "mass": st.mass, "boundary_in": st.boundary_in,
                "alpha_min": st.alpha_min, "alpha_max": st.alpha_max,
                "kernel_launches": st.kernel_launches}

    def profile(self, enable=True, only=None):
        """Enables per-kernel event timing (of kernel name `only`, or of every kernel)."""
        only_id = -1
        if only is not None:
            names = kernel_names()
            only_id = names.index(only)
        self._check(lib().mdbs_profile_enable(self.h, 1 if enable else 0, only_id))

    def profile_read(self):
        """{kernel name: (total device ms, timed launches)} since profiling was enabled."""
        out = {}
        for i in range(lib().mdbs_profile_count()):
            nm, ms, cnt = C.c_char_p(), C.c_double(), C.c_int64()
            self._check(lib().mdbs_profile_read(self.h, i, C.byref(nm), C.byref(ms), C.byref(cnt)))
            if cnt.value:
                out[nm.value.decode()] = (ms.value, cnt.value)
        return out

    def array(self, name):
        n = lib().mdbs_debug_array(self.h, name.encode(), None, 0)
        if n < 0:
            raise KeyError(name)
        out = np.zeros(n)
        lib().mdbs_debug_array(self.h, name.encode(), _ptr(out), n)
        return out

    def set_stream(self, stream_handle: int):
        self._check(lib().mdbs_set_stream(self.h, C.c_void_p(stream_handle)))

    def set_tuning(self, tuning):
        self._check(lib().mdbs_set_tuning(self.h, C.byref(_tuning(tuning))))

    def tuning(self):
        t = Tuning()
        self._check(lib().mdbs_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    def autotune(self, trial_steps=2):
        """Times real steps under candidate schedules and keeps the fastest; the state is
        restored, so the simulation continues as if this had not run.  Returns
        (chosen schedule, [ms per step of each trial])."""
        return _autotune(lib().mdbs_autotune, self.h, trial_steps, self._check)

    def close(self):
        if getattr(self, "h", None):
            lib().mdbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autotune(fn, h, trial_steps, check):
    chosen = Tuning()
    ms = np.zeros(32)
    n = C.c_int32()
    check(fn(h, int(trial_steps), C.byref(chosen), _ptr(ms), len(ms), C.byref(n)))
    return chosen.as_dict(), [float(v) for v in ms[: min(n.value, len(ms))]]


class Batch:
    """Member simulations advanced together, one launch per step phase (mdbs_batch_*)."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (C.c_void_p * len(self.sims))(*[s.h.value if isinstance(s.h, C.c_void_p) else s.h
                                              for s in self.sims])
        h = C.c_void_p()
        rc = lib().mdbs_batch_create(arr, len(self.sims), C.byref(h))
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_batch_last_error(None).decode())
        self.h = h

    def step(self, n=1):
        rc = lib().mdbs_batch_step(self.h, int(n))
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_batch_last_error(self.h).decode())

    def add(self, sim):
        """mdbs_batch_add: sim joins the batch before the next step."""
        rc = lib().mdbs_batch_add(self.h, sim.h)
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_batch_last_error(self.h).decode())
        self.sims.append(sim)

    def remove(self, sim):
        """mdbs_batch_remove: sim leaves the batch and can be stepped alone again."""
        rc = lib().mdbs_batch_remove(self.h, sim.h)
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_batch_last_error(self.h).decode())
        self.sims.remove(sim)

    def set_stream(self, stream_handle: int):
        lib().mdbs_batch_set_stream(self.h, C.c_void_p(stream_handle))

    def _check(self, rc):
        if rc != OK:
            raise MdbsError(rc, lib().mdbs_batch_last_error(self.h).decode())

    def set_tuning(self, tuning):
        self._check(lib().mdbs_batch_set_tuning(self.h, C.byref(_tuning(tuning))))

    def tuning(self):
        t = Tuning()
        self._check(lib().mdbs_batch_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    def autotune(self, trial_steps=1):
        return _autotune(lib().mdbs_batch_autotune, self.h, trial_steps, self._check)

    def close(self):
        if getattr(self, "h", None):
            lib().mdbs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_allocator(alloc=None, free=None):
    """mdbs_set_allocator: alloc(nbytes) -> device address (int, 256-byte aligned, 0 on
    failure) and free(address) serve the arenas of later Simulations; no arguments
    restores cudaMalloc.  The callables are kept alive here until replaced."""
    global _hook
    if alloc is None and free is None:
        rc = lib().mdbs_set_allocator(ALLOC_FN(), FREE_FN(), None)
        _hook = None
    else:
        a = ALLOC_FN(lambda n, ctx: alloc(int(n)) or None)
        f = FREE_FN(lambda p, ctx: free(int(p)))
        rc = lib().mdbs_set_allocator(a, f, None)
        if rc == OK:
            _hook = (a, f)
    if rc != OK:
        raise MdbsError(rc, "mdbs_set_allocator")


def use_torch_allocator():
    """Serve the arenas from PyTorch's caching allocator on the current device."""
    import torch
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n), torch.cuda.caching_allocator_delete)

"""ctypes wrapper of the C oracle (test infrastructure only; see oracle/oracle.h).

Only tests, ``__graft_entry__.smoke()`` and bench.py's cpu_baseline / reference
leg use this module.  It takes a plain case description (grid, fluids,
closures, options, fields) and runs the oracle's own copy of the discrete step.
"""
import ctypes as C

import numpy as np

from .build import build_oracle

_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
        ("rho_l", C.c_double), ("mu_l", C.c_double), ("rho_g", C.c_double), ("mu_g", C.c_double),
        ("sigma", C.c_double), ("g", C.c_double * 3),
        ("kr_model", C.c_int), ("pc_model", C.c_int),
        ("kr_m", C.c_double), ("a_l_irr", C.c_double), ("a_g_irr", C.c_double),
        ("pc0", C.c_double), ("pc_beta", C.c_double), ("pc_m", C.c_double),
        ("a_pc_irr", C.c_double), ("a_pc_max", C.c_double), ("pc_eps", C.c_double),
        ("porous_density", C.c_int), ("theta_deg", C.c_double),
        ("dt", C.c_double), ("cfl", C.c_double), ("dt_max", C.c_double),
        ("c_alpha", C.c_double), ("p_tol", C.c_double),
        ("n_corr", C.c_int), ("mom_sweeps", C.c_int), ("max_cg", C.c_int),
        ("mg_nu1", C.c_int), ("mg_nu2", C.c_int), ("mg_coarse_sweeps", C.c_int),
        ("bc", C.c_int * 6), ("inlet_u", C.c_double), ("inlet_alpha", C.c_double),
    ]


class OrcStats(C.Structure):
    _fields_ = [
        ("steps", C.c_long), ("time", C.c_double), ("dt", C.c_double),
        ("cg_iters", C.c_int * 8), ("cg_resid", C.c_double * 8), ("cg_iters_total", C.c_long),
        ("not_converged", C.c_int), ("mass", C.c_double), ("boundary_in", C.c_double),
        ("alpha_min", C.c_double), ("alpha_max", C.c_double),
    ]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcParams), _D, _D]
        L.orc_set_fields.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_fields.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        L.orc_get_stats.argtypes = [C.c_void_p, C.POINTER(OrcStats)]
        L.orc_get_array.argtypes = [C.c_void_p, C.c_char_p, _D]
        L.orc_get_array.restype = C.c_long
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_closures.argtypes = [C.POINTER(OrcParams), C.c_double, C.c_double, _D]
        L.orc_apply_A.argtypes = [C.c_int] * 3 + [_D] * 6
        L.orc_vcycle.argtypes = [C.c_int] * 3 + [_D] * 4 + [C.c_int] * 3 + [_D, _D]
        L.orc_pcg.argtypes = [C.c_int] * 3 + [_D] * 4 + [C.c_int] * 3 + [_D, _D, C.c_double, C.c_int, _D]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def params_from_case(case) -> OrcParams:
    p = OrcParams()
    for name, _ in OrcParams._fields_:
        if name in ("g", "bc"):
            continue
        setattr(p, name, getattr(case, name))
    p.g = (C.c_double * 3)(*case.g)
    p.bc = (C.c_int * 6)(*case.bc)
    return p


class OracleSim:
    """One simulation held by the oracle."""

    def __init__(self, case):
        self.case = case
        self.prm = params_from_case(case)
        self._phi = _f64(case.porosity.ravel())
        self._k = _f64(case.permeability.ravel())
        self.h = lib().orc_create(C.byref(self.prm), _ptr(self._phi), _ptr(self._k))
        if not self.h:
            raise ValueError("oracle rejected the case")
        self.n = (case.nx, case.ny, case.nz)
        self.set_fields(case.alpha, case.ux, case.uy, case.uz, case.p)

    def set_fields(self, alpha, ux, uy, uz, p):
        a = _f64(alpha.ravel())
        x, y = _f64(ux.ravel()), _f64(uy.ravel())
        z = _f64(uz.ravel()) if uz is not None and uz.size else np.zeros(1)
        pp = _f64(p.ravel())
        rc = lib().orc_set_fields(self.h, _ptr(a), _ptr(x), _ptr(y), _ptr(z), _ptr(pp))
        if rc != 0:
            raise ValueError("oracle set_fields rc=%d" % rc)

    def step(self, n=1):
        rc = lib().orc_step(self.h, int(n))
        if rc != 0:
            raise RuntimeError("oracle step rc=%d" % rc)

    def fields(self):
        nx, ny, nz = self.n
        a = np.zeros(nx * ny * nz)
        p = np.zeros(nx * ny * nz)
        ux = np.zeros((nx + 1) * ny * nz)
        uy = np.zeros(nx * (ny + 1) * nz)
        uz = np.zeros(nx * ny * (nz + 1)) if nz > 1 else np.zeros(0)
        lib().orc_get_fields(self.h, _ptr(a), _ptr(ux), _ptr(uy),
                             _ptr(uz) if nz > 1 else None, _ptr(p))
        return {"alpha": a, "ux": ux, "uy": uy, "uz": uz, "p": p}

    def stats(self):
        st = OrcStats()
        lib().orc_get_stats(self.h, C.byref(st))
        return {
            "steps": st.steps, "time": st.time, "dt": st.dt,
            "cg_iters": list(st.cg_iters)[: self.case.n_corr],
            "cg_resid": list(st.cg_resid)[: self.case.n_corr],
            "cg_iters_total": st.cg_iters_total, "not_converged": st.not_converged,
            "mass": st.mass, "boundary_in": st.boundary_in,
            "alpha_min": st.alpha_min, "alpha_max": st.alpha_max,
        }

    def array(self, name):
        n = lib().orc_get_array(self.h, name.encode(), None)
        if n < 0:
            raise KeyError(name)
        out = np.zeros(n)
        lib().orc_get_array(self.h, name.encode(), _ptr(out))
        return out

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def closures(case, alpha, k0):
    """(krl, krg, Ml, Mg, drag, rho*, pc, cf) of a porous cell, Appendix A / Eqs. 37-45."""
    prm = params_from_case(case)
    out = np.zeros(8)
    lib().orc_closures(C.byref(prm), float(alpha), float(k0), _ptr(out))
    return out


def _coef(T):
    return [_f64(t.ravel()) for t in T]


def apply_A(n, Tx, Ty, Tz, Dd, x):
    Tx, Ty, Tz, Dd = _coef((Tx, Ty, Tz, Dd))
    x = _f64(x.ravel())
    y = np.zeros_like(x)
    lib().orc_apply_A(*n, _ptr(Tx), _ptr(Ty), _ptr(Tz), _ptr(Dd), _ptr(x), _ptr(y))
    return y


def vcycle(n, Tx, Ty, Tz, Dd, r, nu1=2, nu2=2, coarse=0):
    Tx, Ty, Tz, Dd = _coef((Tx, Ty, Tz, Dd))
    r = _f64(r.ravel())
    z = np.zeros_like(r)
    lib().orc_vcycle(*n, _ptr(Tx), _ptr(Ty), _ptr(Tz), _ptr(Dd), nu1, nu2, coarse, _ptr(r), _ptr(z))
    return z


def pcg(n, Tx, Ty, Tz, Dd, b, x0=None, tol=1e-12, max_it=500, nu1=2, nu2=2, coarse=0):
    Tx, Ty, Tz, Dd = _coef((Tx, Ty, Tz, Dd))
    b = _f64(b.ravel())
    x = np.zeros_like(b) if x0 is None else _f64(x0.ravel()).copy()
    res = C.c_double(0)
    it = lib().orc_pcg(*n, _ptr(Tx), _ptr(Ty), _ptr(Tz), _ptr(Dd), nu1, nu2, coarse,
                       _ptr(b), _ptr(x), tol, max_it, C.byref(res))
    return x, it, res.value

"""ctypes binding of the CPU oracle — TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
import this package.  It never imports the product package and the product
never imports it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, EBADSTATE = 0, -1, -4
BC_OUTFLOW, BC_REFLECT, BC_PERIODIC, BC_PREFILLED = 0, 1, 2, 3


class Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("grav", ctypes.c_double * 3),
        ("small_dens", ctypes.c_double),
        ("small_pres", ctypes.c_double),
        ("flatten", ctypes.c_int),
        ("wave_speeds", ctypes.c_int),
        ("grav_energy", ctypes.c_int),
    ]


class Debug(ctypes.Structure):
    _fields_ = [
        ("prim", ctypes.POINTER(ctypes.c_double)),
        ("trace_m", ctypes.POINTER(ctypes.c_double) * 3),
        ("trace_p", ctypes.POINTER(ctypes.c_double) * 3),
        ("flux1", ctypes.POINTER(ctypes.c_double) * 3),
        ("flux_final", ctypes.POINTER(ctypes.c_double) * 3),
    ]


_libs = {}
_D = ctypes.POINTER(ctypes.c_double)


def _lib(counting=False):
    name = "liboracle_count.so" if counting else "liboracle.so"
    if name not in _libs:
        out = _build.build()
        _libs[name] = load(os.path.join(out, name), counting)
    return _libs[name]


def load(path, counting=False):
    """Open an oracle shared library at `path` and declare its entry points."""
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(Params)
    lib.oracle_grown_size.argtypes = [P]
    lib.oracle_grown_size.restype = ctypes.c_longlong
    lib.oracle_fill_ghosts.argtypes = [_D, P]
    lib.oracle_dt.argtypes = [_D, P, _D]
    lib.oracle_step.argtypes = [_D, _D, P, ctypes.c_double, ctypes.POINTER(Debug)]
    lib.oracle_mol_step.argtypes = [_D, _D, P, ctypes.c_int, ctypes.c_double]
    lib.oracle_hllc.argtypes = [_D, _D, ctypes.c_int, ctypes.c_double, _D]
    lib.oracle_wave_speeds.argtypes = [_D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int, _D]
    lib.oracle_ppm_parabola.argtypes = [_D, ctypes.c_double, _D]
    lib.oracle_flatten.argtypes = [_D, _D, ctypes.c_double]
    lib.oracle_flatten.restype = ctypes.c_double
    lib.oracle_integ.argtypes = [_D, ctypes.c_double, ctypes.c_int]
    lib.oracle_integ.restype = ctypes.c_double
    lib.oracle_trace_lines.argtypes = [_D, ctypes.c_int, P, ctypes.c_double, ctypes.c_double, _D, _D]
    lib.oracle_cons_to_prim.argtypes = [_D, P, _D, ctypes.POINTER(ctypes.c_int)]
    lib.oracle_prim_to_cons.argtypes = [_D, ctypes.c_double, _D]
    lib.oracle_exact_star.argtypes = [_D, _D, ctypes.c_double, _D]
    lib.oracle_exact_sample.argtypes = [_D, _D, ctypes.c_double, _D, ctypes.c_int, _D]
    if counting:
        lib.oracle_tally_reset.argtypes = []
        lib.oracle_tally_get.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
        lib.oracle_tally_stages.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    return lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def params(dim, n, dx=None, bc=BC_OUTFLOW, gamma=1.4, cfl=0.5, grav=(0.0, 0.0, 0.0),
           small_dens=1e-200, small_pres=1e-200, flatten=True, einfeldt=False, flux_grav_energy=False):
    """Build a Params struct.  n: interior (nx, ny[, nz]); bc: one kind for
    every face, or a 3x2 nested sequence."""
    n = tuple(n) + (1,) * (3 - len(n))
    if dx is None:
        dx = (1.0 / n[0],) * 3
    P = Params()
    P.dim = dim
    for a in range(3):
        P.n[a] = n[a]
        P.dx[a] = dx[a]
        P.grav[a] = grav[a]
        for s in range(2):
            P.bc[a][s] = bc if isinstance(bc, int) else bc[a][s]
    P.gamma, P.cfl = gamma, cfl
    P.small_dens, P.small_pres = small_dens, small_pres
    P.flatten = 1 if flatten else 0
    P.wave_speeds = 1 if einfeldt else 0
    P.grav_energy = 1 if flux_grav_energy else 0
    return P


def fill_ghosts(U, P):
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    rc = _lib().oracle_fill_ghosts(_ptr(U), ctypes.byref(P))
    if rc:
        raise ValueError(f"oracle_fill_ghosts: {rc}")
    return U


def dt(U, P):
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = ctypes.c_double(0.0)
    rc = _lib().oracle_dt(_ptr(U), ctypes.byref(P), ctypes.byref(out))
    return out.value, rc


def step(U, P, dt_, debug=False):
    """One CTU-PPM step.  Returns (U_new, rc[, intermediates dict])."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    dbg = None
    arrs = None
    if debug:
        N = U[0].size
        arrs = {"prim": np.zeros((6,) + U.shape[1:])}
        for key in ("trace_m", "trace_p", "flux1", "flux_final"):
            arrs[key] = [np.zeros_like(U) for _ in range(3)]
        dbg = Debug()
        dbg.prim = _ptr(arrs["prim"])
        for key in ("trace_m", "trace_p", "flux1", "flux_final"):
            for d in range(3):
                getattr(dbg, key)[d] = _ptr(arrs[key][d])
    rc = _lib().oracle_step(_ptr(U), _ptr(out), ctypes.byref(P), float(dt_),
                            ctypes.byref(dbg) if dbg is not None else None)
    if rc == EINVAL:
        raise ValueError("oracle_step: invalid arguments")
    if debug:
        return out, rc, arrs
    return out, rc


def mol_step(U, P, dt_):
    """One method-of-lines step (SSP-RK2, PPM edges, HLLC) of a state with
    U.shape[0] - 5 passive species.  Returns (U_new, rc)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    rc = _lib().oracle_mol_step(_ptr(U), _ptr(out), ctypes.byref(P), U.shape[0] - 5, float(dt_))
    if rc == EINVAL:
        raise ValueError("oracle_mol_step: invalid arguments")
    return out, rc


def run(U, P, nsteps, dt_fixed=None):
    """Advance nsteps with the oracle's own CFL dt (or a fixed dt).  Returns (U, t, dts)."""
    t, dts = 0.0, []
    for _ in range(nsteps):
        if dt_fixed is None:
            d, rc = dt(U, P)
            if rc:
                raise RuntimeError(f"oracle_dt: bad state ({rc})")
        else:
            d = dt_fixed
        U, rc = step(U, P, d)
        if rc:
            raise RuntimeError(f"oracle_step: bad state ({rc})")
        t += d
        dts.append(d)
    return U, t, dts


def count_ops(U, P, dt_):
    """Algorithmic FP64 operation tally of one step: dict(add, mul, div, sqrt, cmp)."""
    lib = _lib(counting=True)
    lib.oracle_tally_reset()
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    lib.oracle_step(_ptr(U), _ptr(out), ctypes.byref(P), float(dt_), None)
    t = (ctypes.c_longlong * 5)()
    lib.oracle_tally_get(t)
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), list(t)))


STAGES = ("prim", "trace", "flux1", "flux2", "flux3", "update")


def count_ops_by_stage(U, P, dt_):
    """Per-stage operation tallies of one step: {stage: dict(add, mul, div, sqrt, cmp)}."""
    lib = _lib(counting=True)
    lib.oracle_tally_reset()
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty_like(U)
    lib.oracle_step(_ptr(U), _ptr(out), ctypes.byref(P), float(dt_), None)
    t = (ctypes.c_longlong * 30)()
    lib.oracle_tally_stages(t)
    keys = ("add", "mul", "div", "sqrt", "cmp")
    return {st: dict(zip(keys, list(t)[5 * k: 5 * k + 5])) for k, st in enumerate(STAGES)}


def hllc(qL, qR, d, gamma):
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    F = np.zeros(5)
    _lib().oracle_hllc(_ptr(qL), _ptr(qR), d, gamma, _ptr(F))
    return F


def wave_speeds(qL, qR, d, gamma, einfeldt):
    out = np.zeros(2)
    _lib().oracle_wave_speeds(_ptr(np.ascontiguousarray(qL, dtype=np.float64)),
                              _ptr(np.ascontiguousarray(qR, dtype=np.float64)), d, gamma, 1 if einfeldt else 0,
                              _ptr(out))
    return out


def ppm_parabola(line7, chi=1.0):
    a = np.ascontiguousarray(line7, dtype=np.float64)
    out = np.zeros(3)
    _lib().oracle_ppm_parabola(_ptr(a), chi, _ptr(out))
    return out  # am, ap, a6


def flatten_coef(p7, un7, small_pres=1e-200):
    return _lib().oracle_flatten(_ptr(np.ascontiguousarray(p7, dtype=np.float64)),
                                 _ptr(np.ascontiguousarray(un7, dtype=np.float64)), small_pres)


def integ(am_ap_a6, sigma, plus):
    return _lib().oracle_integ(_ptr(np.ascontiguousarray(am_ap_a6, dtype=np.float64)), sigma, 1 if plus else 0)


def trace_lines(lines6x7, d, P, dtdx, dt_):
    L = np.ascontiguousarray(lines6x7, dtype=np.float64)
    qm, qp = np.zeros(5), np.zeros(5)
    _lib().oracle_trace_lines(_ptr(L), d, ctypes.byref(P), dtdx, dt_, _ptr(qm), _ptr(qp))
    return qm, qp


def cons_to_prim(U5, P):
    U5 = np.ascontiguousarray(U5, dtype=np.float64)
    q = np.zeros(5)
    bad = ctypes.c_int(0)
    _lib().oracle_cons_to_prim(_ptr(U5), ctypes.byref(P), _ptr(q), ctypes.byref(bad))
    return q, bad.value


def prim_to_cons(q5, gamma):
    q5 = np.ascontiguousarray(q5, dtype=np.float64)
    U = np.zeros(5)
    _lib().oracle_prim_to_cons(_ptr(q5), gamma, _ptr(U))
    return U


def exact_star(WL, WR, gamma):
    out = np.zeros(2)
    rc = _lib().oracle_exact_star(_ptr(np.asarray(WL, dtype=np.float64)),
                                  _ptr(np.asarray(WR, dtype=np.float64)), gamma, _ptr(out))
    if rc:
        raise ValueError("vacuum")
    return out[0], out[1]


def exact_sample(WL, WR, gamma, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    W = np.zeros((xi.size, 3))
    rc = _lib().oracle_exact_sample(_ptr(np.asarray(WL, dtype=np.float64)),
                                    _ptr(np.asarray(WR, dtype=np.float64)), gamma, _ptr(xi), xi.size, _ptr(W))
    if rc:
        raise ValueError("vacuum")
    return W

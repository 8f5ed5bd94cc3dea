"""CPU FP64 oracle (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It wraps ``kn_oracle.c`` (plain C,
FP64, loops in reaction-index order, no FMA contraction) through ctypes and
shares no code with the CUDA library.  See the header of ``kn_oracle.c`` for
which passage of the paper each function follows and how each is pinned.

The learned-timestep pieces (features, MLP forward/backward) live in
``oracle/mlp.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

STATUS = {0: "ok", 1: "step_limit", 2: "dt_underflow", 3: "nonfinite", 4: "max_reject"}


def build(force: bool = False) -> str:
    """Compile kn_oracle.c into liboracle.so next to it (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Net(C.Structure):
    _fields_ = [("N", C.c_int32), ("R", C.c_int32), ("A", C.c_void_p), ("reac", C.c_void_p),
                ("prod", C.c_void_p), ("ln_k0", C.c_void_p), ("t9_exp", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("kappa", C.c_double), ("eps_r", C.c_double), ("eps_c", C.c_double),
                ("y_min", C.c_double), ("grow_max", C.c_double), ("safety", C.c_double),
                ("shrink", C.c_double), ("max_reject", C.c_int32), ("method", C.c_int32),
                ("max_steps", C.c_int64), ("dt_min_frac", C.c_double)]


class _Zone(C.Structure):
    _fields_ = [("T0", C.c_double), ("rho0", C.c_double), ("tau", C.c_double),
                ("t_start", C.c_double), ("t_end", C.c_double), ("dt_trial", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_next", C.c_double), ("steps", C.c_int64),
                ("rejects", C.c_int64), ("status", C.c_int32), ("pad", C.c_int32)]


@dataclass
class OracleOpts:
    kappa: float = 1.0
    eps_r: float = 0.05
    eps_c: float = 1e-6
    y_min: float = 1e-10
    grow_max: float = 1.5
    safety: float = 0.9
    shrink: float = 0.5
    max_reject: int = 60
    max_steps: int = 10_000_000
    dt_min_frac: float = 1e-30
    method: int = 0  # 0: Eq. (3) with the kappa switch; 1: alpha-QSS (METHOD_QSS)

    def c(self) -> _Opts:
        return _Opts(self.kappa, self.eps_r, self.eps_c, self.y_min, self.grow_max, self.safety,
                     self.shrink, self.max_reject, self.method, self.max_steps, self.dt_min_frac)


METHOD_ASYMPTOTIC, METHOD_QSS = 0, 1


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_rates.argtypes = [C.POINTER(_Net), C.c_double, C.c_double, P]
        L.or_rhs.argtypes = [C.POINTER(_Net), P, P, P, P, P]
        L.or_update.argtypes = [C.c_int, P, P, P, C.c_double, C.c_double, P, P]
        L.or_test.argtypes = [C.c_int, P, P, P, C.POINTER(_Opts), P, P, P]
        L.or_test.restype = C.c_int
        L.or_growth.argtypes = [C.c_double, C.c_double, C.POINTER(_Opts)]
        L.or_growth.restype = C.c_double
        L.or_conditions.argtypes = [C.c_double] * 4 + [P, P]
        L.or_integrate.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.POINTER(_Zone), P,
                                   C.POINTER(_Result), P, C.c_int64]
        L.or_replay.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.POINTER(_Zone), P, P,
                                C.c_int64, P]
        L.or_integrate_batch.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.c_int32, P, P, P,
                                         C.c_int32]
        L.or_be_step.argtypes = [C.POINTER(_Net), P, P, C.c_double, P, C.c_double, C.c_double,
                                 C.c_int]
        L.or_be_step.restype = C.c_int
        L.or_be_fixed.argtypes = [C.POINTER(_Net), C.POINTER(_Zone), P, C.c_int64, C.c_double,
                                  C.c_double, C.c_int]
        L.or_be_fixed.restype = C.c_int
        L.or_be_integrate.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.POINTER(_Zone), P,
                                      C.POINTER(_Result), C.c_int]
        L.or_be_integrate_batch.argtypes = [C.POINTER(_Net), C.POINTER(_Opts), C.c_int32, P, P,
                                            P, C.c_int32, C.c_int32]
        L.or_qss_alpha.argtypes = [C.c_double]
        L.or_qss_alpha.restype = C.c_double
        L.or_qss_predict.argtypes = [C.c_int, P, P, P, C.c_double, P]
        L.or_qss_correct.argtypes = [C.c_int, P, P, P, P, P, C.c_double, P]
        L.or_lu_solve.argtypes = [C.c_int, P, P]
        L.or_lu_solve.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


class Oracle:
    """Oracle bound to one network (keeps the arrays alive for ctypes)."""

    def __init__(self, net):
        self.net = net
        self.N = net.n_species
        self.R = net.n_reactions
        self._A = _f64(net.A)
        self._reac = np.ascontiguousarray(net.reac, dtype=np.int32)
        self._prod = np.ascontiguousarray(net.prod, dtype=np.int32)
        self._lnk = _f64(net.ln_k0)
        self._n = _f64(net.t9_exp)
        self.cnet = _Net(self.N, self.R, _p(self._A).value, _p(self._reac).value,
                         _p(self._prod).value, _p(self._lnk).value, _p(self._n).value)

    # ---- single pieces ---------------------------------------------------
    def conditions(self, T0, rho0, tau, t):
        a, b = C.c_double(), C.c_double()
        lib().or_conditions(T0, rho0, tau, t, C.byref(a), C.byref(b))
        return a.value, b.value

    def rates(self, T9, rho):
        k = np.empty(self.R)
        lib().or_rates(C.byref(self.cnet), T9, rho, _p(k))
        return k

    def rhs(self, k, Y):
        k, Y = _f64(k), _f64(Y)
        Fp, kk, f = np.empty(self.N), np.empty(self.N), np.empty(self.R)
        lib().or_rhs(C.byref(self.cnet), _p(k), _p(Y), _p(Fp), _p(kk), _p(f))
        return Fp, kk, f

    def update(self, Y, Fp, kk, dt, kappa=1.0):
        Y, Fp, kk = _f64(Y), _f64(Fp), _f64(kk)
        Yn = np.empty(self.N)
        asy = np.empty(self.N, dtype=np.int8)
        lib().or_update(self.N, _p(Y), _p(Fp), _p(kk), dt, kappa, _p(Yn), _p(asy))
        return Yn, asy.astype(bool)

    def test(self, Y, Yn, opts: OracleOpts | None = None):
        o = (opts or OracleOpts()).c()
        Y, Yn = _f64(Y), _f64(Yn)
        cons, rel, fin = C.c_double(), C.c_double(), C.c_int()
        acc = lib().or_test(self.N, _p(self._A), _p(Y), _p(Yn), C.byref(o), C.byref(cons),
                            C.byref(rel), C.byref(fin))
        return bool(acc), cons.value, rel.value, bool(fin.value)

    def growth(self, rel, cons, opts: OracleOpts | None = None):
        o = (opts or OracleOpts()).c()
        return lib().or_growth(rel, cons, C.byref(o))

    def step(self, Y, T9, rho, dt, kappa=1.0):
        """One kappa-switched update from Y at (T9, rho): returns Y', asy mask."""
        k = self.rates(T9, rho)
        Fp, kk, _ = self.rhs(k, Y)
        return self.update(Y, Fp, kk, dt, kappa)

    # ---- the alpha-QSS update (Sec. 11's alternative to Eq. 3) ----------
    @staticmethod
    def qss_alpha(x):
        return lib().or_qss_alpha(float(x))

    def qss_predict(self, Y, Fp, kk, dt):
        Y, Fp, kk = _f64(Y), _f64(Fp), _f64(kk)
        Yp = np.empty(self.N)
        lib().or_qss_predict(self.N, _p(Y), _p(Fp), _p(kk), dt, _p(Yp))
        return Yp

    def qss_correct(self, Y, Fp0, k0, Fpp, kp, dt):
        Y, Fp0, k0, Fpp, kp = map(_f64, (Y, Fp0, k0, Fpp, kp))
        Yc = np.empty(self.N)
        lib().or_qss_correct(self.N, _p(Y), _p(Fp0), _p(k0), _p(Fpp), _p(kp), dt, _p(Yc))
        return Yc

    def qss_step(self, Y, T9, rho, dt, T9p=None, rhop=None):
        """One alpha-QSS step from Y: rates at (T9, rho) for the start state and
        at (T9p, rhop) (default: the same) for the predicted one.  Returns
        (Y', F+0, k0, Yp)."""
        k = self.rates(T9, rho)
        Fp0, k0, _ = self.rhs(k, Y)
        Yp = self.qss_predict(Y, Fp0, k0, dt)
        kq = k if T9p is None else self.rates(T9p, rhop)
        Fpp, kp, _ = self.rhs(kq, Yp)
        return self.qss_correct(Y, Fp0, k0, Fpp, kp, dt), Fp0, k0, Yp

    # ---- whole integrations --------------------------------------------
    @staticmethod
    def _zone(zones, z):
        return _Zone(float(zones.T0[z]), float(zones.rho0[z]), float(zones.tau[z]),
                     float(zones.t_start[z]), float(zones.t_end[z]), float(zones.dt_trial[z]))

    def integrate(self, zones, z=0, opts: OracleOpts | None = None, record: int = 0, Y0=None):
        """Integrate zone z.  Returns dict(Y, t, dt_next, steps, rejects, status[, dts])."""
        o = (opts or OracleOpts()).c()
        Y = _f64(zones.Y0[z] if Y0 is None else Y0).copy()
        res = _Result()
        rec = np.empty(record) if record else None
        lib().or_integrate(C.byref(self.cnet), C.byref(o), C.byref(self._zone(zones, z)), _p(Y),
                           C.byref(res), _p(rec) if record else None, int(record))
        out = dict(Y=Y, t=res.t, dt_next=res.dt_next, steps=res.steps, rejects=res.rejects,
                   status=res.status)
        if record:
            out["dts"] = rec[: min(res.steps, record)].copy()
        return out

    def replay(self, zones, z, dts, opts: OracleOpts | None = None):
        o = (opts or OracleOpts()).c()
        Y = _f64(zones.Y0[z]).copy()
        dts = _f64(dts)
        t = C.c_double()
        lib().or_replay(C.byref(self.cnet), C.byref(o), C.byref(self._zone(zones, z)), _p(Y),
                        _p(dts), len(dts), C.byref(t))
        return Y, t.value

    def integrate_batch(self, zones, opts: OracleOpts | None = None, threads: int = 1):
        o = (opts or OracleOpts()).c()
        Z = zones.n_zones
        czones = (_Zone * Z)(*[self._zone(zones, z) for z in range(Z)])
        Y = _f64(zones.Y0).copy()
        res = (_Result * Z)()
        lib().or_integrate_batch(C.byref(self.cnet), C.byref(o), Z, C.cast(czones, C.c_void_p),
                                 _p(Y), C.cast(res, C.c_void_p), threads)
        return _results(Y, res)

    def be_step(self, k, Y0, dt, tol=1e-14, y_floor=1e-30, max_iter=50):
        Y0 = _f64(Y0)
        Y = np.empty(self.N)
        it = lib().or_be_step(C.byref(self.cnet), _p(_f64(k)), _p(Y0), dt, _p(Y), tol, y_floor,
                              max_iter)
        return Y, it

    def be_fixed(self, zones, z, n_steps, tol=1e-14, y_floor=1e-30, max_iter=50):
        Y = _f64(zones.Y0[z]).copy()
        it = lib().or_be_fixed(C.byref(self.cnet), C.byref(self._zone(zones, z)), _p(Y),
                               int(n_steps), tol, y_floor, max_iter)
        return Y, it

    def be_integrate(self, zones, z=0, opts: OracleOpts | None = None, max_iter=6):
        o = (opts or OracleOpts()).c()
        Y = _f64(zones.Y0[z]).copy()
        res = _Result()
        lib().or_be_integrate(C.byref(self.cnet), C.byref(o), C.byref(self._zone(zones, z)),
                              _p(Y), C.byref(res), max_iter)
        return dict(Y=Y, t=res.t, dt_next=res.dt_next, steps=res.steps, rejects=res.rejects,
                    status=res.status)

    def be_integrate_batch(self, zones, opts: OracleOpts | None = None, max_iter=6, threads=1):
        o = (opts or OracleOpts()).c()
        Z = zones.n_zones
        czones = (_Zone * Z)(*[self._zone(zones, z) for z in range(Z)])
        Y = _f64(zones.Y0).copy()
        res = (_Result * Z)()
        lib().or_be_integrate_batch(C.byref(self.cnet), C.byref(o), Z, C.cast(czones, C.c_void_p),
                                    _p(Y), C.cast(res, C.c_void_p), max_iter, threads)
        return _results(Y, res)


def _results(Y, res):
    return dict(
        Y=Y,
        t=np.array([r.t for r in res]),
        dt_next=np.array([r.dt_next for r in res]),
        steps=np.array([r.steps for r in res], dtype=np.int64),
        rejects=np.array([r.rejects for r in res], dtype=np.int64),
        status=np.array([r.status for r in res], dtype=np.int32),
    )


def lu_solve(J, b):
    """Dense LU solve from the oracle (for pinning the LU itself)."""
    J = _f64(J).copy()
    x = _f64(b).copy()
    rc = lib().or_lu_solve(int(J.shape[0]), _p(J), _p(x))
    if rc != 0:
        raise ZeroDivisionError("singular matrix")
    return x

"""ctypes binding of the one-dimensional C oracle (``ch_oracle.c``). TEST INFRASTRUCTURE ONLY.

Functions and the passages they follow:

* ``dh_apply``       D_h of Eq. 3.2 (Dirichlet, h = 1/(n+1)).
* ``band_solve``     Gaussian elimination with partial pivoting (textbook, banded storage).
* ``step``           one step of Eq. 2.4 (LIN1), Eq. 2.3 + Newton Eq. 3.17/3.18 (NL), Eq. 2.5 (LIN2).
* ``propagate``      repeated steps; optional manufactured forcing (test support).
* ``fine_solution``  sequential fine solve, the serial method Parareal converges to.
* ``parareal``       Eq. 2.2 with the coarse initial guess and stop rule of Section 4.
* ``energy``         discrete form of Eq. 1.2.

Pins (tests/test_oracle_1d.py): D_h eigenvalues against the formula under Eq. 3.2; dense
brute-force solves; manufactured solutions at first order in time and second in space
(Section 2.1); frozen-coefficient steps and Parareal iterates against the closed forms
of Lemma 3.1 and Lemma 3.4; finite-step convergence (Theorem 3.7, remark at the end of
Section 3); energy decay of the Eyre scheme (Section 2.1, Eq. 1.3).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

LIN1, NL, LIN2 = 0, 1, 2
SCHEMES = {"lin1": LIN1, "nl": NL, "lin2": LIN2}

_lib = None


class _Params(C.Structure):
    _fields_ = [("n", C.c_int), ("eps", C.c_double), ("T", C.c_double), ("N", C.c_int),
                ("J", C.c_int), ("coarse_steps", C.c_int), ("fine_scheme", C.c_int),
                ("coarse_scheme", C.c_int), ("newton_tol", C.c_double), ("newton_max", C.c_int),
                ("frozen", C.c_int), ("tol", C.c_double), ("max_iters", C.c_int), ("newton_form", C.c_int)]


class _Forcing(C.Structure):
    _fields_ = [("nmodes", C.c_int), ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("m", C.POINTER(C.c_int))]


class _Stats(C.Structure):
    _fields_ = [("newton_total", C.c_longlong), ("newton_max_seen", C.c_int), ("steps", C.c_longlong)]


class _Result(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("inc", C.c_double * 1024),
                ("err_l2", C.c_double * 1024), ("err_max", C.c_double * 1024), ("st", _Stats)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build())
        d = C.POINTER(C.c_double)
        _lib.orc1d_dh_apply.argtypes = [C.c_int, d, d]
        _lib.orc_band_solve.argtypes = [C.c_int, C.c_int, C.c_int, d, d]
        _lib.orc1d_step.argtypes = [C.POINTER(_Params), C.c_int, C.c_double, C.c_double, d, d,
                                    C.POINTER(_Forcing), C.POINTER(_Stats)]
        _lib.orc1d_propagate.argtypes = [C.POINTER(_Params), C.c_int, C.c_double, C.c_int, C.c_double,
                                         d, d, C.POINTER(_Forcing), C.POINTER(_Stats)]
        _lib.orc1d_fine_solution.argtypes = [C.POINTER(_Params), d, d, C.POINTER(_Stats)]
        _lib.orc1d_parareal.argtypes = [C.POINTER(_Params), d, d, d, C.POINTER(_Result)]
        _lib.orc1d_energy.argtypes = [C.c_int, C.c_double, d]
        _lib.orc1d_energy.restype = C.c_double
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Problem and method parameters (Section 2, Section 4)."""
    n: int
    eps: float
    T: float
    N: int
    J: int
    coarse_steps: int = 1
    fine: str = "lin1"
    coarse: str = "lin1"
    newton_tol: float = 1e-12
    newton_max: int = 50
    frozen: bool = False
    tol: float = 0.0
    max_iters: int = -1
    newton_form: int = 0  # 0: Eq. 3.18 as printed, direct linear steps; 1: Y - J^{-1} H(Y) for all (other rounding)

    def c(self) -> _Params:
        mi = self.N if self.max_iters < 0 else self.max_iters
        return _Params(self.n, self.eps, self.T, self.N, self.J, self.coarse_steps, SCHEMES[self.fine],
                       SCHEMES[self.coarse], self.newton_tol, self.newton_max, int(self.frozen),
                       self.tol, mi, self.newton_form)


@dataclass
class PararealResult:
    U: np.ndarray
    iterations: int
    converged: bool
    inc: np.ndarray
    err_l2: np.ndarray = field(default_factory=lambda: np.zeros(0))
    err_max: np.ndarray = field(default_factory=lambda: np.zeros(0))
    newton_total: int = 0
    newton_max: int = 0
    steps: int = 0


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc} "
                          "(1 invalid argument, 2 singular pivot, 3 Newton not converged)")


def dh_apply(u) -> np.ndarray:
    u = _f64(u)
    out = np.empty_like(u)
    _check(lib().orc1d_dh_apply(u.size, _ptr(u), _ptr(out)), "dh_apply")
    return out


def band_solve(ab: np.ndarray, b, kl: int, ku: int) -> np.ndarray:
    """ab: n x (2kl+ku+1) band rows (row i holds columns i-kl .. i+kl+ku)."""
    ab = _f64(ab).copy()
    x = _f64(b).copy()
    _check(lib().orc_band_solve(x.size, kl, ku, _ptr(ab), _ptr(x)), "band_solve")
    return x


def _forcing(modes):
    if not modes:
        return None, None
    a = _f64([m[0] for m in modes])
    b = _f64([m[1] for m in modes])
    mm = np.ascontiguousarray([m[2] for m in modes], dtype=np.int32)
    f = _Forcing(len(modes), _ptr(a), _ptr(b), mm.ctypes.data_as(C.POINTER(C.c_int)))
    return f, (a, b, mm)


def step(p: Params, scheme: str, dt: float, u, t_next: float = 0.0, forcing=None):
    u = _f64(u)
    out = np.empty_like(u)
    st = _Stats()
    f, keep = _forcing(forcing)
    cp = p.c()
    _check(lib().orc1d_step(C.byref(cp), SCHEMES[scheme], dt, t_next, _ptr(u), _ptr(out),
                            C.byref(f) if f else None, C.byref(st)), "step")
    return out, st.newton_total


def propagate(p: Params, scheme: str, dt: float, nsteps: int, u, t0: float = 0.0, forcing=None):
    """forcing: list of (a, b, m) giving g(x,t) = sum a e^{b t} sin(m pi x)."""
    u = _f64(u)
    out = np.empty_like(u)
    st = _Stats()
    f, keep = _forcing(forcing)
    cp = p.c()
    _check(lib().orc1d_propagate(C.byref(cp), SCHEMES[scheme], dt, nsteps, t0, _ptr(u), _ptr(out),
                                 C.byref(f) if f else None, C.byref(st)), "propagate")
    return out


def fine_solution(p: Params, u0) -> np.ndarray:
    u0 = _f64(u0)
    Uf = np.empty((p.N + 1, p.n))
    st = _Stats()
    cp = p.c()
    _check(lib().orc1d_fine_solution(C.byref(cp), _ptr(u0), _ptr(Uf), C.byref(st)), "fine_solution")
    return Uf


def parareal(p: Params, u0, Ufine=None) -> PararealResult:
    u0 = _f64(u0)
    U = np.empty((p.N + 1, p.n))
    res = _Result()
    cp = p.c()
    uf = _f64(Ufine) if Ufine is not None else None
    _check(lib().orc1d_parareal(C.byref(cp), _ptr(u0), _ptr(uf) if uf is not None else None, _ptr(U),
                                C.byref(res)), "parareal")
    k = res.iterations
    return PararealResult(U=U, iterations=k, converged=bool(res.converged),
                            inc=np.array(res.inc[:k]),
                            err_l2=np.array(res.err_l2[:k + 1]) if uf is not None else np.zeros(0),
                            err_max=np.array(res.err_max[:k + 1]) if uf is not None else np.zeros(0),
                            newton_total=res.st.newton_total, newton_max=res.st.newton_max_seen,
                            steps=res.st.steps)


def energy(u, eps: float) -> float:
    u = _f64(u)
    return lib().orc1d_energy(u.size, eps, _ptr(u))

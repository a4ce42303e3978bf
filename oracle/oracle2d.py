"""Two-dimensional CPU oracle (numpy/scipy, FP64). TEST INFRASTRUCTURE ONLY.

Omega = (0,1)^2 with n x n interior nodes (x_i, y_j) = (i h, j h), h = 1/(n+1), stored
row-major (y outer, x inner); boundary values are zero. The 2D discrete Laplacian is the
natural extension of Eq. 3.2 (the remark closing Section 3): D_h = I (x) D_1 + D_1 (x) I, with
D_1 = h^-2 tridiag(1,-2,1). Each implicit step is the paper's definition solved by a sparse
direct factorisation (SuperLU via scipy, a library solve):

* ``step('lin1')``  Eq. 2.4  (I - dt D_h diag(u^n)^2 + eps^2 dt D_h^2) u^{n+1} = (I - dt D_h) u^n
* ``step('nl')``    Eq. 2.3 by the Newton iteration of Eq. 3.18 from Y_0 = u^n, with the stop
                    rule of the 1D oracle (||dY||_inf <= tol, or the FP64 rounding floor)
* ``step('lin2')``  Eq. 2.5 with D_h on the implicit 2 dt term
* ``Params.solver = 'pcg'``  the same steps with every linear system J x = b solved by library CG
                    (scipy) on the symmetric positive definite A^{-1} J x = A^{-1} b (A = -D_h,
                    A^{-1} applied by the library sine transform, whose basis diagonalises D_h,
                    eigenvalues below Eq. 3.2), two rounds of iterative refinement against the
                    sparse FP64 residual b - J x; for grids where sparse LU takes minutes
* ``parareal``      Eq. 2.2, coarse initial guess (Section 4), correction F + (G_new - G_old)
* ``energy``        discrete Eq. 1.2

Pins (tests/test_oracle_2d.py): eigenvalues of D_h against lambda_p + lambda_q (formula below
Eq. 3.2), dense brute force built from the pinned 1D operator, manufactured solutions (order
1 in time, 2 in space), frozen-coefficient factors (Lemma 3.1) and Parareal closed form
(Lemma 3.4) per sine mode, finite-step exactness, Eyre energy decay; the error norms against
discrete sine orthogonality; the energy against its closed form on a sine mode; the 'pcg'
solver against the sparse direct solves (every scheme, frozen or not).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_CACHE = {}


def dh_matrix(n: int) -> sp.csc_matrix:
    """D_h on the n x n interior grid, row-major (x fastest)."""
    key = ("dh", n)
    if key not in _CACHE:
        h = 1.0 / (n + 1)
        d1 = sp.diags([np.ones(n - 1), -2.0 * np.ones(n), np.ones(n - 1)], [-1, 0, 1], shape=(n, n)) / h ** 2
        eye = sp.identity(n)
        _CACHE[key] = (sp.kron(eye, d1) + sp.kron(d1, eye)).tocsc()
    return _CACHE[key]


def dh2_matrix(n: int) -> sp.csc_matrix:
    key = ("dh2", n)
    if key not in _CACHE:
        D = dh_matrix(n)
        _CACHE[key] = (D @ D).tocsc()
    return _CACHE[key]


def sine_transform(x: np.ndarray) -> np.ndarray:
    """Orthonormal 2D DST-I over the last two axes (scipy.fft, a library FFT): S X S with
    S_jk = sqrt(2/(n+1)) sin(pi j k/(n+1)), the eigenvector basis of D_h (below Eq. 3.2)."""
    import scipy.fft
    return scipy.fft.dstn(np.asarray(x, dtype=np.float64), type=1, axes=(-2, -1), norm="ortho")


def dh_apply(u: np.ndarray, n: int) -> np.ndarray:
    return dh_matrix(n) @ u


@dataclass
class Params:
    n: int
    eps: float
    T: float
    N: int
    J: int
    coarse_steps: int = 1
    fine: str = "nl"
    coarse: str = "lin1"
    newton_tol: float = 1e-12
    newton_max: int = 50
    frozen: bool = False
    tol: float = 0.0
    max_iters: int = -1
    solver: str = "direct"  # "direct": sparse LU; "pcg": library CG on A^{-1} J (large grids)


class OracleError(RuntimeError):
    pass


def _forcing(modes, n, t):
    """g(x,y,t) = sum a e^{b t} sin(mx pi x) sin(my pi y) on the interior grid."""
    if not modes:
        return None
    x = np.arange(1, n + 1) / (n + 1)
    g = np.zeros((n, n))
    for a, b, mx, my in modes:
        g += a * math.exp(b * t) * np.outer(np.sin(my * np.pi * x), np.sin(mx * np.pi * x))
    return g.reshape(-1)


def _cg(op, b, M, rtol=1e-10):
    """Library CG (scipy) to a relative residual of rtol."""
    try:
        x, info = spla.cg(op, b, M=M, rtol=rtol, atol=0.0, maxiter=2000)
    except TypeError:  # scipy before rtol
        x, info = spla.cg(op, b, M=M, tol=rtol, atol=0.0, maxiter=2000)
    if info != 0:
        raise OracleError(f"CG did not converge (info {info})")
    return x


def _solve(p: Params, dt: float, c: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x with (I + eps^2 dt A^2 + dt A diag(c)) x = b, A = -D_h, c >= 0.

    'direct': sparse LU of the assembled matrix. 'pcg': J = A S with S = A^{-1} + eps^2 dt A +
    dt diag(c) symmetric positive definite, so CG on S x = A^{-1} b (relative residual 1e-10)
    with the preconditioner A^{-1} + eps^2 dt A + dt mean(c) I (diagonal in the sine basis),
    then two refinements, each a CG solve for the FP64 residual b - J x of the sparse
    matrices."""
    n = p.n
    D = dh_matrix(n)
    e2 = p.eps ** 2
    if p.solver == "direct":
        J = (sp.identity(n * n, format="csc") + e2 * dt * dh2_matrix(n) - dt * D @ sp.diags(c)).tocsc()
        return spla.splu(J).solve(b)
    lam = -np.add.outer(eigenvalues_1d(n), eigenvalues_1d(n))  # eigenvalues of A, [q][p]
    cbar = float(np.mean(c))
    pre = 1.0 / (1.0 / lam + e2 * dt * lam + dt * cbar)

    def ainv(v):
        return sine_transform(sine_transform(v.reshape(n, n)) / lam).reshape(-1)

    S = spla.LinearOperator((n * n, n * n), matvec=lambda v: ainv(v) - e2 * dt * (D @ v) + dt * c * v,
                            dtype=np.float64)
    M = spla.LinearOperator((n * n, n * n), matvec=lambda v: sine_transform(
        sine_transform(v.reshape(n, n)) * pre).reshape(-1), dtype=np.float64)

    def jmul(v):
        Av = -(D @ v)
        return v - e2 * dt * (D @ Av) + dt * (-(D @ (c * v)))

    x = _cg(S, ainv(b), M)
    for _ in range(2):
        x = x + _cg(S, ainv(b - jmul(x)), M)
    return x


def eigenvalues_1d(n: int) -> np.ndarray:
    """lambda_p = (2/h^2)(cos(p pi h) - 1), p = 1..n: eigenvalues of D_1 (below Eq. 3.2)."""
    h = 1.0 / (n + 1)
    return (2.0 / h ** 2) * (np.cos(np.arange(1, n + 1) * np.pi * h) - 1.0)


def step(p: Params, scheme: str, dt: float, u: np.ndarray, t_next: float = 0.0, forcing=None):
    """One step; returns (u_next, newton_iterations)."""
    n = p.n
    D = dh_matrix(n)
    e2 = p.eps ** 2
    g = _forcing(forcing, n, t_next)
    if scheme == "lin1":
        w = np.ones_like(u) if p.frozen else u * u
        # (I - dt D diag(w) + eps^2 dt D^2) = I + eps^2 dt A^2 + dt A diag(w)
        rhs = u - dt * (D @ u)
        if g is not None:
            rhs = rhs + dt * g
        return _solve(p, dt, w, rhs), 0
    if scheme == "lin2":
        v = u if p.frozen else u ** 3
        # (I - 2 dt D + eps^2 dt D^2) = I + eps^2 dt A^2 + dt A diag(2)
        rhs = u + dt * (D @ v) - 3 * dt * (D @ u)
        if g is not None:
            rhs = rhs + dt * g
        return _solve(p, dt, np.full_like(u, 2.0), rhs), 0
    if scheme == "nl":
        yhat = u - dt * (D @ u)  # Eq. 3.17
        if g is not None:
            yhat = yhat + dt * g
        y = u.copy()
        prev = 0.0
        for m in range(1, p.newton_max + 1):
            if p.frozen:
                nxt = _solve(p, dt, np.ones_like(y), yhat)  # (I + eps^2 dt D^2 - dt D) Y = Yhat
            else:
                w = y * y
                # Eq. 3.18: (I + eps^2 dt D^2 - 3 dt D diag(Y^2)) Y_{m+1} = Yhat - 2 dt D (Y^3)
                nxt = _solve(p, dt, 3.0 * w, yhat - 2 * dt * (D @ (w * y)))
            diff = float(np.max(np.abs(nxt - y)))
            y = nxt
            if diff <= p.newton_tol:
                return y, m
            if m >= 2 and diff <= math.sqrt(p.newton_tol) and diff > 0.5 * prev:
                return y, m  # FP64 rounding floor of the residual
            prev = diff
        raise OracleError("Newton did not converge")
    raise ValueError(scheme)


def propagate(p: Params, scheme: str, dt: float, nsteps: int, u: np.ndarray, t0: float = 0.0, forcing=None):
    y = np.array(u, dtype=np.float64)
    for s in range(nsteps):
        y, _ = step(p, scheme, dt, y, t0 + (s + 1) * dt, forcing)
    return y


def fine(p: Params, u):
    return propagate(p, p.fine, p.T / p.N / p.J, p.J, u)


def coarse(p: Params, u):
    return propagate(p, p.coarse, p.T / p.N / p.coarse_steps, p.coarse_steps, u)


def fine_solution(p: Params, u0) -> np.ndarray:
    U = np.empty((p.N + 1, p.n * p.n))
    U[0] = u0
    for s in range(p.N):
        U[s + 1] = fine(p, U[s])
    return U


@dataclass
class PararealResult:
    U: np.ndarray
    iterations: int
    converged: bool
    inc: np.ndarray
    err_l2: np.ndarray = field(default_factory=lambda: np.zeros(0))
    err_max: np.ndarray = field(default_factory=lambda: np.zeros(0))


def _errors(U, Uf, h):
    d = U - Uf
    return float(np.max(np.sqrt(h * h * np.sum(d * d, axis=1)))), float(np.max(np.abs(d)))


def _fine_of(args):
    p, u = args
    return fine(p, u)


def parareal(p: Params, u0, Ufine=None, max_iters=None, pmap=map) -> PararealResult:
    """Eq. 2.2 with the coarse initial guess; stop on max_n ||U^k - U^{k-1}||_inf < tol.
    pmap: the map applied to the slices' fine propagations of an iteration (e.g. a process pool's
    map; the slices are independent, which is the parallelism Parareal exposes)."""
    N = p.N
    mi = (N if p.max_iters < 0 else p.max_iters) if max_iters is None else max_iters
    h = 1.0 / (p.n + 1)
    U = np.empty((N + 1, p.n * p.n))
    U[0] = u0
    Gold = np.empty((N, p.n * p.n))
    for s in range(N):
        U[s + 1] = coarse(p, U[s])
        Gold[s] = U[s + 1]
    inc, el2, emx = [], [], []
    if Ufine is not None:
        a, b = _errors(U, Ufine, h)
        el2.append(a)
        emx.append(b)
    converged = False
    k = 0
    for k in range(1, mi + 1):
        Fk = dict(zip(range(k - 1, N), pmap(_fine_of, [(p, U[s]) for s in range(k - 1, N)])))
        Unew = U.copy()
        for s in range(k - 1, N):
            g = coarse(p, Unew[s])
            Unew[s + 1] = Fk[s] + (g - Gold[s])
            Gold[s] = g
        inc.append(float(np.max(np.abs(Unew - U))))
        U = Unew
        if Ufine is not None:
            a, b = _errors(U, Ufine, h)
            el2.append(a)
            emx.append(b)
        if p.tol > 0 and inc[-1] < p.tol:
            converged = True
            break
    if mi == 0:
        k = 0
    return PararealResult(U=U, iterations=k, converged=converged, inc=np.array(inc), err_l2=np.array(el2),
                          err_max=np.array(emx))


def energy(u: np.ndarray, n: int, eps: float) -> float:
    h = 1.0 / (n + 1)
    D = dh_matrix(n)
    return float(h * h * np.sum((u * u - 1.0) ** 2 / 4.0) + 0.5 * eps ** 2 * h * h * (u @ (-(D @ u))))

"""Neumann-Neumann fine solver of Section 4.6 in 1D (numpy, FP64). TEST INFRASTRUCTURE ONLY.

One step of the linear scheme Eq. 2.4 written in the mixed form of Section 4.6,

    u - dt D v = u^n,        eps^2 D u - c^2 u + v = -u^n,        c^2 = (u^n)^2 (1 if frozen),

(eliminating v gives (I + eps^2 dt D^2 - dt D c^2) u = (I - dt D) u^n, Eq. 2.4), with D the
three-point Laplacian of Eq. 3.2 and u = v = 0 on the boundary, solved by the Neumann-Neumann
iteration over N0 equal subdomains. Discrete reading: the interior nodes 1..n (h = 1/(n+1),
n + 1 = N0 m) are split by the interface nodes k m, k = 1..N0-1; each interface row of the global
system is shared by its two subdomains, the mass-like terms (u, c^2 u, v) half each and the
Laplacian split into its one-sided parts, so that the local matrices sum to the global one.
Starting from interface values (g, h) = (u^n, v(u^n)) at the interfaces, each iteration
  1. solves the Dirichlet problems (interior rows, interface values fixed),
  2. forms the residual of the global rows at the interfaces,
  3. solves the Neumann problems (local matrix with its interface rows, zero data inside, the
     residual on the interface rows),
  4. updates g, h by theta times the sum of the two Neumann solutions at each interface,
until both updates have Euclidean norm over the interfaces <= tol; the step is then the
Dirichlet solution for the last interface values. This is Richardson iteration on the interface
Schur complement with the Neumann-Neumann preconditioner; its fixed point is the global step.
Local systems are solved densely with numpy (a library solve).

Pins (tests/test_oracle_nn.py): the converged step against the C oracle's banded LIN1 step;
the local matrices summing to the global matrix; N0 = 1 (no interface) against the same;
exact convergence after one update for two mirror-symmetric subdomains with theta = 1/4.
"""
from __future__ import annotations

import numpy as np


def global_matrix(n: int, eps: float, dt: float, c2: np.ndarray) -> np.ndarray:
    """The mixed system's matrix, unknowns interleaved (u_1, v_1, u_2, v_2, ...)."""
    h2 = (1.0 / (n + 1)) ** 2
    A = np.zeros((2 * n, 2 * n))
    for j in range(n):
        A[2 * j, 2 * j] = 1.0
        A[2 * j, 2 * j + 1] = 2.0 * dt / h2
        A[2 * j + 1, 2 * j] = -2.0 * eps ** 2 / h2 - c2[j]
        A[2 * j + 1, 2 * j + 1] = 1.0
        for nb in (j - 1, j + 1):
            if 0 <= nb < n:
                A[2 * j, 2 * nb + 1] = -dt / h2
                A[2 * j + 1, 2 * nb] = eps ** 2 / h2
    return A


def local_matrix(n: int, eps: float, dt: float, c2: np.ndarray, lo: int, hi: int, left_if: bool,
                 right_if: bool) -> np.ndarray:
    """Local matrix of the subdomain with nodes lo..hi (0-based, inclusive); the end nodes that are
    interfaces (left_if, right_if) carry their half of the global row."""
    h2 = (1.0 / (n + 1)) ** 2
    m = hi - lo + 1
    A = np.zeros((2 * m, 2 * m))
    for r in range(m):
        j = lo + r
        half = (r == 0 and left_if) or (r == m - 1 and right_if)
        s = 0.5 if half else 1.0
        # mass-like terms
        A[2 * r, 2 * r] = s
        A[2 * r + 1, 2 * r] = -s * c2[j]
        A[2 * r + 1, 2 * r + 1] = s
        # Laplacian couplings to the neighbours inside this subdomain (one-sided at an interface)
        for nb in (r - 1, r + 1):
            if 0 <= nb < m:
                A[2 * r, 2 * nb + 1] += -dt / h2
                A[2 * r, 2 * r + 1] += dt / h2
                A[2 * r + 1, 2 * nb] += eps ** 2 / h2
                A[2 * r + 1, 2 * r] += -eps ** 2 / h2
        # a physical boundary next to this node keeps the full diagonal (u = v = 0 there)
        if j == 0 or j == n - 1:
            A[2 * r, 2 * r + 1] += dt / h2
            A[2 * r + 1, 2 * r] += -eps ** 2 / h2
    return A


def nn_step(n: int, eps: float, dt: float, un: np.ndarray, N0: int, theta: float = 0.25, tol: float = 1e-10,
            max_iter: int = 200, frozen: bool = False):
    """One step of Eq. 2.4 by the Neumann-Neumann iteration; returns (u^{n+1}, iterations)."""
    un = np.asarray(un, dtype=np.float64)
    if (n + 1) % N0:
        raise ValueError("n + 1 must be a multiple of the subdomain count")
    m = (n + 1) // N0
    h2 = (1.0 / (n + 1)) ** 2
    c2 = np.ones(n) if frozen else un * un
    f = np.empty(2 * n)
    f[0::2] = un
    f[1::2] = -un
    A = global_matrix(n, eps, dt, c2)
    if N0 == 1:
        x = np.linalg.solve(A, f)
        return x[0::2].copy(), 0
    gam = [k * m - 1 for k in range(1, N0)]  # 0-based interface nodes
    # initial interface values: u^n and v computed from u^n by the second equation
    lap = np.zeros(n)
    for j in range(n):
        lap[j] = ((un[j - 1] if j > 0 else 0.0) - 2.0 * un[j] + (un[j + 1] if j < n - 1 else 0.0)) / h2
    v0 = -un - eps ** 2 * lap + c2 * un
    G = np.zeros(2 * n)  # full vector; only interface entries are used as data
    for g in gam:
        G[2 * g], G[2 * g + 1] = un[g], v0[g]
    subs = [(i * m, (i + 1) * m - 2) for i in range(N0)]  # interior nodes of each subdomain

    def dirichlet(G):
        x = G.copy()
        for lo, hi in subs:
            idx = np.arange(2 * lo, 2 * hi + 2)
            rhs = f[idx] - A[np.ix_(idx, np.setdiff1d(np.arange(2 * n), idx))] @ G[np.setdiff1d(np.arange(2 * n), idx)]
            x[idx] = np.linalg.solve(A[np.ix_(idx, idx)], rhs)
        for g in gam:
            x[2 * g], x[2 * g + 1] = G[2 * g], G[2 * g + 1]
        return x

    it = 0
    while True:
        x = dirichlet(G)
        r = f - A @ x  # zero on the interior rows; the interface residual on the interface rows
        upd = np.zeros(2 * n)
        for i, (lo, hi) in enumerate(subs):
            a = lo - 1 if i > 0 else lo
            b = hi + 1 if i < N0 - 1 else hi
            L = local_matrix(n, eps, dt, c2, a, b, i > 0, i < N0 - 1)
            rhs = np.zeros(2 * (b - a + 1))
            if i > 0:
                rhs[0:2] = r[2 * a:2 * a + 2]
            if i < N0 - 1:
                rhs[-2:] = r[2 * b:2 * b + 2]
            w = np.linalg.solve(L, rhs)
            if i > 0:
                upd[2 * a:2 * a + 2] += w[0:2]
            if i < N0 - 1:
                upd[2 * b:2 * b + 2] += w[-2:]
        it += 1
        dg = np.array([theta * upd[2 * g] for g in gam])
        dh = np.array([theta * upd[2 * g + 1] for g in gam])
        for g in gam:
            G[2 * g] += theta * upd[2 * g]
            G[2 * g + 1] += theta * upd[2 * g + 1]
        if (np.linalg.norm(dg) <= tol and np.linalg.norm(dh) <= tol) or it >= max_iter:
            break
    x = dirichlet(G)
    return x[0::2].copy(), it


def nn_propagate(n: int, eps: float, dt: float, nsteps: int, u, N0: int, theta: float = 0.25, tol: float = 1e-10,
                 max_iter: int = 200, frozen: bool = False):
    """nsteps steps of nn_step; returns (u, total iterations)."""
    u = np.asarray(u, dtype=np.float64).copy()
    total = 0
    for _ in range(nsteps):
        u, it = nn_step(n, eps, dt, u, N0, theta, tol, max_iter, frozen)
        total += it
    return u, total

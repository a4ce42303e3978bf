"""A-priori Parareal error bounds of Section 3 (numpy, FP64). TEST INFRASTRUCTURE ONLY.

The convergence theorems of Section 3 bound the Parareal error of iterate k by a factor times
the error of the coarse initial guess:

    max_j ||E_j^k|| <= a^k min{ ((1 - b^(N-1)) / (1 - b))^k , C(N-1, k) } max_j ||E_j^0||

* PA-I  (Theorem 3.7):  a = ||P_J1 - P_1||, b = ||P_1||
* PA-II (Theorem 3.9):  a = ||P_J2 - P_2||, b = ||P_2||
* PA-III (Theorem 3.11): a = ||P_J2 - P_1||, b = ||P_1||
* NPA-I (Theorem 3.16): a = C_1 dT^2, b = ||P_1||;  NPA-II (Theorem 3.21): a = C_2 dT^2,
  b = ||P_3|| (C_1, C_2 are LTE constants the paper fits to measurements; the caller gives them)

with P_i = (I - i dT D_h + eps^2 dT D_h^2)^-1 (I - i dT D_h) (the frozen propagators, Section 3)
and P_Ji the same with dT / J applied J times. The norm is the Euclidean 2-norm; every P is a
rational function of the symmetric D_h, so its norm is the largest modulus over the eigenvalues
of D_h: lambda_p = -(4/h^2) sin^2(p pi / (2(n+1))) in 1D (formula below Eq. 3.2), and
lambda_p + lambda_q on the 2D grid. With y = -lambda, the factor of P_i on a mode is
g_i(y) = (1 + i dT y) / (1 + i dT y + eps^2 dT y^2) (Lemma 3.1).

Readings: the fine factor of a mode is the eigenvalue of P_Ji as the matrix is defined, the
J-th power of (1 + i dt y) / (1 + i dt y + eps^2 dt y^2) with dt = dT / J (Lemma 3.2 abbreviates
it as g_i(y/J)^J, which would scale the eps^2 term by 1/J^2 instead of 1/J). With
coarse_steps = m coarse steps per slice, the coarse propagator is P_i(dT/m)^m and its norm
replaces ||P_i|| in a and b (the paper uses m = 1).

Pins (tests/test_oracle_bounds.py): the norms against dense matrices built from D_h and
taken through numpy's matrix inverse, power and 2-norm (1D and 2D); Lemma 3.1 and Lemma 3.2
ranges; the binomial branch making the factor 0 for k >= N; and the bound holding for the
oracle's own frozen Parareal iterates.
"""
from __future__ import annotations

import math

import numpy as np

# (fine i, coarse i) of the propagators P_i in each variant's bound
VARIANT_FACTORS = {"PA-I": (1, 1), "PA-II": (2, 2), "PA-III": (2, 1), "NPA-I": (None, 1), "NPA-II": (None, 3)}


def eigen_y(n: int, dim: int) -> np.ndarray:
    """-lambda for every eigenvalue lambda of D_h (1D: n values, 2D: n^2 values)."""
    h = 1.0 / (n + 1)
    p = np.arange(1, n + 1)
    mu = 4.0 / h ** 2 * np.sin(p * np.pi / (2.0 * (n + 1))) ** 2
    if dim == 1:
        return mu
    return (mu[:, None] + mu[None, :]).reshape(-1)


def g(i: int, step: float, eps: float, y):
    """Lemma 3.1: factor of (I - i s D_h + eps^2 s D_h^2)^-1 (I - i s D_h) on the mode -lambda = y."""
    return (1.0 + i * step * y) / (1.0 + i * step * y + eps ** 2 * step * y ** 2)


def norms(variant: str, n: int, dim: int, eps: float, T: float, N: int, J: int, coarse_steps: int = 1):
    """(a, b) of the variant's bound; a is None for the nonlinear variants (a = C dT^2)."""
    fi, ci = VARIANT_FACTORS[variant]
    y = eigen_y(n, dim)
    dT = T / N
    coarse = g(ci, dT / coarse_steps, eps, y) ** coarse_steps
    b = float(np.max(np.abs(coarse)))
    if fi is None:
        return None, b
    fine = g(fi, dT / J, eps, y) ** J
    return float(np.max(np.abs(fine - coarse))), b


def factors(a: float, b: float, N: int, kmax: int) -> np.ndarray:
    """The bound's factor for k = 0..kmax: a^k min{((1 - b^(N-1)) / (1 - b))^k, C(N-1, k)}."""
    out = np.zeros(kmax + 1)
    s = (1.0 - b ** (N - 1)) / (1.0 - b)
    for k in range(kmax + 1):
        c = math.comb(N - 1, k) if k <= N - 1 else 0
        out[k] = a ** k * min(s ** k, c)
    return out


def bound(variant: str, n: int, dim: int, eps: float, T: float, N: int, J: int, kmax: int,
          lte_const: float = 0.0, coarse_steps: int = 1):
    """(a, b, factors[0..kmax]); for NPA-I / NPA-II, a = lte_const * dT^2."""
    a, b = norms(variant, n, dim, eps, T, N, J, coarse_steps)
    if a is None:
        if not lte_const > 0:
            raise ValueError("the nonlinear variants need the LTE constant")
        a = lte_const * (T / N) ** 2
    return a, b, factors(a, b, N, kmax)

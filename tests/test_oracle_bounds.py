"""Pins of the Section 3 bound oracle (oracle/bounds.py), CPU only.

The per-mode formulas are checked against dense matrices (the propagators built from D_h by
matrix inverse and power, their 2-norms by SVD), so a wrong eigenvalue, a swapped fine/coarse
factor, a dt where dT belongs or a missing power of J fails here; the bound itself is checked
against the oracle's own frozen Parareal iterates.
"""
import math

import numpy as np
import pytest

import ch_inputs
from oracle import bounds as ob
from oracle import oracle1d as o


def dense_dh(n: int, dim: int) -> np.ndarray:
    h = 1.0 / (n + 1)
    d1 = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2
    if dim == 1:
        return d1
    eye = np.eye(n)
    return np.kron(eye, d1) + np.kron(d1, eye)


def dense_prop(D, i, step, eps, m=1):
    eye = np.eye(D.shape[0])
    one = np.linalg.solve(eye - i * step * D + eps ** 2 * step * D @ D, eye - i * step * D)
    return np.linalg.matrix_power(one, m)


@pytest.mark.parametrize("dim,n", [(1, 12), (1, 31), (2, 5)])
@pytest.mark.parametrize("variant", ["PA-I", "PA-II", "PA-III"])
@pytest.mark.parametrize("coarse_steps", [1, 3])
def test_norms_match_dense_matrices(dim, n, variant, coarse_steps):
    eps, T, N, J = 0.0725, 1.0, 8, 20
    D = dense_dh(n, dim)
    fi, ci = ob.VARIANT_FACTORS[variant]
    dT = T / N
    Pc = dense_prop(D, ci, dT / coarse_steps, eps, coarse_steps)
    PJ = dense_prop(D, fi, dT / J, eps, J)
    a_ref = np.linalg.norm(PJ - Pc, 2)
    b_ref = np.linalg.norm(Pc, 2)
    a, b = ob.norms(variant, n, dim, eps, T, N, J, coarse_steps)
    assert abs(a - a_ref) <= 1e-10 * a_ref
    assert abs(b - b_ref) <= 1e-12


@pytest.mark.parametrize("variant,ci", [("NPA-I", 1), ("NPA-II", 3)])
def test_nonlinear_variants_use_the_coarse_linearisation(variant, ci):
    n, eps, T, N = 16, 0.05, 0.5, 10
    D = dense_dh(n, 1)
    b_ref = np.linalg.norm(dense_prop(D, ci, T / N, eps), 2)
    a, b, f = ob.bound(variant, n, 1, eps, T, N, 100, 5, lte_const=0.1181)
    assert abs(b - b_ref) <= 1e-12
    assert a == pytest.approx(0.1181 * (T / N) ** 2, rel=1e-15)
    with pytest.raises(ValueError):
        ob.bound(variant, n, 1, eps, T, N, 100, 5)


def test_lemma_3_1_and_3_2_ranges():
    """g_i in (0, 1) for y > 0 (Lemma 3.1); |fine - coarse| < 1 (Lemma 3.2), hence a, b < 1."""
    y = np.logspace(-3, 9, 400)
    for i in (1, 2, 3):
        gi = ob.g(i, 0.01, 0.05, y)
        assert np.all((gi > 0) & (gi < 1))
    for variant in ("PA-I", "PA-II", "PA-III"):
        for eps in (0.0725, 0.725):
            a, b = ob.norms(variant, 63, 1, eps, 1.0, 20, 200)
            assert 0 < a < 1 and 0 < b < 1


def test_factor_is_one_at_k0_and_zero_from_k_equal_n():
    """The binomial branch: C(N-1, k) = 0 for k >= N (finite-step convergence)."""
    a, b = 0.3, 0.97
    N = 6
    f = ob.factors(a, b, N, 9)
    assert f[0] == 1.0
    assert np.all(f[N:] == 0.0)
    s = (1 - b ** (N - 1)) / (1 - b)
    for k in range(1, N):
        assert f[k] == pytest.approx(a ** k * min(s ** k, math.comb(N - 1, k)), rel=1e-15)


@pytest.mark.parametrize("fine,coarse,variant", [("lin1", "lin1", "PA-I"), ("lin2", "lin2", "PA-II"),
                                                 ("lin2", "lin1", "PA-III")])
def test_bound_holds_for_oracle_frozen_parareal(fine, coarse, variant):
    """Theorems 3.7 / 3.9 / 3.11 on the frozen model: the oracle's Parareal errors (Euclidean
    norm, maximum over slices) stay below factor_k times the error of the coarse initial guess."""
    n, eps, T, N, J = 31, 0.0725, 1.0, 10, 20
    u0 = ch_inputs.initial_condition(1, n, 11, amp=0.5)
    base = dict(n=n, eps=eps, T=T, N=N, J=J, fine=fine, coarse=coarse, frozen=True)
    Uf = o.fine_solution(o.Params(**base), u0)
    _, _, f = ob.bound(variant, n, 1, eps, T, N, J, N)
    errs = []
    for k in range(0, N + 1):
        r = o.parareal(o.Params(**base, max_iters=k), u0, Uf)
        errs.append(max(np.linalg.norm(r.U[j] - Uf[j]) for j in range(1, N + 1)))
    assert errs[0] > 0
    for k in range(1, N + 1):
        assert errs[k] <= f[k] * errs[0] * (1 + 1e-9) + 1e-13, (k, errs[k], f[k] * errs[0])

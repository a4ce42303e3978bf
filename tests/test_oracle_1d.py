"""Pins of the one-dimensional CPU oracle against facts the paper and mathematics fix.

Each test below would fail under a plausible mistake in the oracle: a wrong D_h scale or
sign (eigenvalues), a transposed D_h diag(w) (manufactured-solution order), a dropped
eps^2 term or a wrong coarse/fine factor (closed forms of Lemma 3.1 / Lemma 3.4), a wrong
sign or index in the Parareal correction (closed form, finite-step exactness), or a
non-converged Newton (residual and energy decay).
"""
import math

import numpy as np
import pytest

import ch_inputs
from oracle import oracle1d as o


def dense_dh(n):
    """D_h as a dense matrix, probed column by column through the oracle."""
    eye = np.eye(n)
    return np.stack([o.dh_apply(eye[:, j]) for j in range(n)], axis=1)


def sine_mode(n, p):
    x = np.arange(1, n + 1) / (n + 1)
    return np.sin(p * np.pi * x)


def mu(n, p):
    """-lambda_p, lambda_p = (2/h^2)(cos(p pi/(N_x - 1)) - 1), N_x = n + 2 (below Eq. 3.2)."""
    h = 1.0 / (n + 1)
    return -(2.0 / h ** 2) * (math.cos(p * math.pi / (n + 1)) - 1.0)


# ------------------------------------------------------------------------- D_h


@pytest.mark.parametrize("n", [5, 16, 33])
def test_dh_eigenvalues_match_paper_formula(n):
    D = dense_dh(n)
    assert np.allclose(D, D.T, rtol=0, atol=0)
    ev = np.sort(np.linalg.eigvalsh(D))
    lam = np.sort([-mu(n, p) for p in range(1, n + 1)])
    assert np.max(np.abs(ev - lam) / np.abs(lam)) < 1e-12
    assert np.all(ev < 0)


def test_dh_sine_modes_are_eigenvectors():
    n = 40
    for p in (1, 7, 40):
        v = sine_mode(n, p)
        assert np.allclose(o.dh_apply(v), -mu(n, p) * v, rtol=0, atol=1e-9 * mu(n, p))


# ---------------------------------------------------------------- banded solver


def test_band_solve_matches_dense_with_pivoting():
    rng = np.random.default_rng(3)
    n, kl, ku = 30, 2, 2
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            A[i, j] = rng.standard_normal()
    A[np.arange(n), np.arange(n)] *= 1e-3  # forces row exchanges
    b = rng.standard_normal(n)
    w = 2 * kl + ku + 1
    ab = np.zeros((n, w))
    for i in range(n):
        for j in range(max(0, i - kl), min(n, i + ku + 1)):
            ab[i, j - i + kl] = A[i, j]
    x = o.band_solve(ab, b, kl, ku)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------ single time steps


def dense_step(scheme, u, dt, eps):
    n = u.size
    D = dense_dh(n)
    I = np.eye(n)
    if scheme == "lin1":
        A = I - dt * D @ np.diag(u ** 2) + eps ** 2 * dt * D @ D
        return np.linalg.solve(A, u - dt * D @ u)
    if scheme == "lin2":
        A = I - 2 * dt * D + eps ** 2 * dt * D @ D
        return np.linalg.solve(A, u + dt * D @ u ** 3 - 3 * dt * D @ u)
    raise ValueError(scheme)


@pytest.mark.parametrize("scheme", ["lin1", "lin2"])
def test_linear_steps_match_dense_brute_force(scheme):
    n, eps, dt = 14, 0.1, 1e-3
    u = ch_inputs.initial_condition(1, n, 5, amp=0.8)
    p = o.Params(n=n, eps=eps, T=1, N=1, J=1)
    out, _ = o.step(p, scheme, dt, u)
    ref = dense_step(scheme, u, dt, eps)
    assert np.max(np.abs(out - ref)) < 1e-12


def test_newton_step_solves_nonlinear_system():
    """Newton result is a root of H(Y) = Y + eps^2 dt D^2 Y - dt D Y^3 - (I - dt D) u (Eq. 3.17)."""
    n, eps, dt = 16, 0.1, 5e-3
    u = ch_inputs.initial_condition(1, n, 6, amp=0.9)
    p = o.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13)
    y, iters = o.step(p, "nl", dt, u)
    D = dense_dh(n)
    H = y + eps ** 2 * dt * D @ D @ y - dt * D @ y ** 3 - (u - dt * D @ u)
    scale = np.max(np.abs(eps ** 2 * dt * D @ D @ y)) + 1
    assert np.max(np.abs(H)) < 1e-12 * scale
    assert 2 <= iters <= 8


def _dh_extended(v, n):
    """D_h (Eq. 3.2, zero Dirichlet values) in numpy's extended precision."""
    w = np.zeros(n + 2, dtype=np.longdouble)
    w[1:-1] = v
    return (w[:-2] - 2 * w[1:-1] + w[2:]) * np.longdouble((n + 1) ** 2)


@pytest.mark.parametrize("n,eps,dt,amp,tol", [
    (1024, 0.02, 1.0 / (64 * 200), 0.1, 1e-12),  # the 1D nonlinear workload's grid and fine step
    (1024, 0.02, 1.0 / (64 * 200), 0.9, 1e-12),  # same, states near the wells: the floor exit decides
    (255, 0.02, 1e-4, 0.9, 1e-10),
    (63, 0.1, 1e-3, 0.9, 1e-12),
])
def test_newton_stops_at_the_root_within_the_rounding_floor(n, eps, dt, amp, tol):
    """Where Newton stops, by the increment test or by the rounding-floor exit (an increment
    below sqrt(tol) that fails to halve), the step is the root of Eq. 3.17 to within
    max(tol, u * 16 eps^2 dt / h^4 * max|Y|): one Newton correction with the residual evaluated
    in extended precision moves it by no more. An exit that accepted a slowly converging
    iterate (up to sqrt(tol) = 1e-6 here) would fail this."""
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended precision on this platform")
    u = ch_inputs.initial_condition(1, n, 3, amp=amp)
    y, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=tol), "nl", dt, u)
    Y, U, dtl = y.astype(np.longdouble), u.astype(np.longdouble), np.longdouble(dt)
    H = (Y + np.longdouble(eps) ** 2 * dtl * _dh_extended(_dh_extended(Y, n), n) - dtl * _dh_extended(Y ** 3, n)
         - (U - dtl * _dh_extended(U, n)))
    D = dense_dh(n)
    Jac = np.eye(n) + eps ** 2 * dt * D @ D - 3 * dt * D @ np.diag(y ** 2)
    dist = np.max(np.abs(np.linalg.solve(Jac, H.astype(np.float64))))
    floor = np.finfo(np.float64).eps * 16 * eps ** 2 * dt * (n + 1) ** 4 * np.max(np.abs(y))
    assert dist <= max(tol, floor), (dist, tol, floor)


def test_newton_forms_reach_the_same_root():
    """Eq. 3.18 as printed and the unsimplified Newton step give the same step to rounding."""
    n, eps, dt = 40, 0.1, 2e-3
    u = ch_inputs.initial_condition(1, n, 7, amp=0.9)
    a, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13), "nl", dt, u)
    b, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13, newton_form=1), "nl", dt, u)
    assert np.max(np.abs(a - b)) < 1e-13


@pytest.mark.parametrize("scheme", ["lin1", "lin2"])
@pytest.mark.parametrize("frozen", [False, True])
def test_linear_steps_from_their_residual_match_dense_brute_force(scheme, frozen):
    """The residual form of the linear steps (Eq. 2.4 / 2.5 reached by Y <- Y - M^{-1} H(Y) from
    u^n) is the same step as the direct solve: both against a dense solve, to rounding; the
    iteration stops after a few refinements."""
    n, eps, dt = 14, 0.1, 1e-3
    u = ch_inputs.initial_condition(1, n, 5, amp=0.8)
    p = o.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13, newton_form=1, frozen=frozen)
    out, iters = o.step(p, scheme, dt, u)
    if frozen:
        D, I = dense_dh(n), np.eye(n)
        c = 1.0 if scheme == "lin1" else 2.0
        rhs = u - dt * D @ u if scheme == "lin1" else u + dt * D @ u - 3 * dt * D @ u
        ref = np.linalg.solve(I - c * dt * D + eps ** 2 * dt * D @ D, rhs)
    else:
        ref = dense_step(scheme, u, dt, eps)
    assert np.max(np.abs(out - ref)) < 1e-12
    direct, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1, frozen=frozen), scheme, dt, u)
    assert np.max(np.abs(out - direct)) < 1e-13
    assert 1 <= iters <= 4


@pytest.mark.parametrize("scheme,i", [("lin1", 1), ("lin2", 2), ("nl", 1)])
def test_frozen_step_matches_lemma_3_1_factor(scheme, i):
    """Frozen model (diag(u^2) = I): each sine mode is scaled by g_i(mu_p) of Lemma 3.1."""
    n, eps, dt = 31, 0.07, 2e-3
    p = o.Params(n=n, eps=eps, T=1, N=1, J=1, frozen=True)
    for pm in (1, 5, 31):
        v = sine_mode(n, pm)
        out, _ = o.step(p, scheme, dt, v)
        y = mu(n, pm)
        g = (1 + i * dt * y) / (1 + i * dt * y + eps ** 2 * dt * y ** 2)
        assert 0 < g < 1
        assert np.max(np.abs(out - g * v)) < 1e-13


# ------------------------------------------------------- manufactured solutions


def mms_forcing(eps):
    """u = e^{-t} sin(pi x) solves u_t + eps^2 D^2 u = D(u^3 - u) + g with this g."""
    pi2 = np.pi ** 2
    return [(-1 + eps ** 2 * pi2 ** 2 - pi2, -1.0, 1), (0.75 * pi2, -3.0, 1), (-2.25 * pi2, -3.0, 3)]


def mms_error(scheme, n, nsteps, T, eps=0.1):
    x = np.arange(1, n + 1) / (n + 1)
    u0 = np.sin(np.pi * x)
    p = o.Params(n=n, eps=eps, T=T, N=1, J=nsteps, newton_tol=1e-13)
    uT = o.propagate(p, scheme, T / nsteps, nsteps, u0, forcing=mms_forcing(eps))
    return np.max(np.abs(uT - math.exp(-T) * u0))


@pytest.mark.parametrize("scheme", ["nl", "lin1", "lin2"])
def test_mms_first_order_in_time(scheme):
    errs = [mms_error(scheme, 511, m, 0.2) for m in (40, 80, 160)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2, errs


@pytest.mark.parametrize("scheme", ["nl", "lin1"])
def test_mms_second_order_in_space(scheme):
    errs = [mms_error(scheme, n, 2000, 0.02) for n in (15, 31, 63)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, errs


# ----------------------------------------------------------------- energy decay


def test_eyre_scheme_energy_non_increasing_at_large_steps():
    """The nonlinear scheme Eq. 2.3 is unconditionally gradient stable (Section 2.1)."""
    n, eps = 63, 0.04
    u = ch_inputs.initial_condition(1, n, 11, amp=0.5)
    p = o.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13)
    E = [o.energy(u, eps)]
    for dt in [1e-3] * 5 + [2e-2] * 5 + [0.5] * 3:
        u, _ = o.step(p, "nl", dt, u)
        E.append(o.energy(u, eps))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1])), np.diff(E)
    assert E[-1] < E[0]


def test_energy_matches_definition_on_sine():
    n, eps = 50, 0.3
    v = 0.5 * sine_mode(n, 2)
    h = 1.0 / (n + 1)
    bulk = h * np.sum((v ** 2 - 1) ** 2 / 4)
    grad = 0.5 * eps ** 2 * h * mu(n, 2) * np.sum(v ** 2)  # v^T(-D_h)v = mu_p |v|^2
    assert abs(o.energy(v, eps) - (bulk + grad)) < 1e-12


# -------------------------------------------------------------------- Parareal


def frozen_parareal_closed_form(n, p_mode, eps, T, N, J, k):
    """Lemma 3.4 / proof of Theorem 3.7 per DST mode: U_s^k = sum_{j<=k} C(s,j)(b-a)^j a^{s-j} u0."""
    y = mu(n, p_mode)
    dT = T / N
    dt = dT / J
    a = (1 + dT * y) / (1 + dT * y + eps ** 2 * dT * y ** 2)
    b = ((1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)) ** J
    coef = np.array([sum(math.comb(s, j) * (b - a) ** j * a ** (s - j) for j in range(min(k, s) + 1))
                     for s in range(N + 1)])
    return coef


@pytest.mark.parametrize("k", [0, 1, 2, 5, 8])
def test_frozen_parareal_matches_closed_form(k):
    n, eps, T, N, J = 31, 0.0725, 1.0, 8, 20
    pm = 3
    p = o.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1", frozen=True, max_iters=k)
    u0 = sine_mode(n, pm)
    r = o.parareal(p, u0)
    coef = frozen_parareal_closed_form(n, pm, eps, T, N, J, k)
    expect = coef[:, None] * u0[None, :]
    assert r.iterations == k
    assert np.max(np.abs(r.U - expect)) < 1e-12


def test_frozen_parareal_error_within_theorem_3_7_bound():
    n, eps, T, N, J = 31, 0.0725, 1.0, 10, 20
    u0 = sum(sine_mode(n, pm) / pm for pm in range(1, n + 1))
    p = o.Params(n=n, eps=eps, T=T, N=N, J=J, frozen=True)
    Uf = o.fine_solution(p, u0)
    dT, dt = T / N, T / N / J
    ys = np.array([mu(n, pm) for pm in range(1, n + 1)])
    P1 = (1 + dT * ys) / (1 + dT * ys + eps ** 2 * dT * ys ** 2)
    PJ = ((1 + dt * ys) / (1 + dt * ys + eps ** 2 * dt * ys ** 2)) ** J
    alpha, beta = np.max(np.abs(PJ - P1)), np.max(np.abs(P1))  # 2-norms of symmetric operators
    E0 = None
    for k in range(0, N):
        r = o.parareal(o.Params(n=n, eps=eps, T=T, N=N, J=J, frozen=True, max_iters=k), u0)
        e = max(np.linalg.norm(r.U[j] - Uf[j]) for j in range(1, N + 1))
        if k == 0:
            E0 = e
            continue
        bound = alpha ** k * min(((1 - beta ** (N - 1)) / (1 - beta)) ** k, math.comb(N - 1, k)) * E0
        assert e <= bound * (1 + 1e-9) + 1e-14


@pytest.mark.parametrize("fine", ["lin1", "nl"])
def test_parareal_finite_step_exactness(fine):
    """U_s^k equals the sequential fine solution for s <= k, and everywhere at k = N."""
    n, N = 32, 6
    u0 = ch_inputs.initial_condition(1, n, 2, amp=0.3)
    p = o.Params(n=n, eps=0.08, T=0.2, N=N, J=10, fine=fine, coarse="lin1")
    Uf = o.fine_solution(p, u0)
    for k in range(0, N + 1):
        r = o.parareal(o.Params(**{**p.__dict__, "max_iters": k}), u0, Uf)
        assert np.array_equal(r.U[: k + 1], Uf[: k + 1])
    assert r.err_max[-1] == 0.0


def test_parareal_stop_rule_on_paper_e1_parameters():
    """Section 4.1 parameters (T=1, h=1/64, N=20, J=200, eps=0.0725) with a smooth u0.

    The stop rule halts at the first iteration whose increment is below tol; the error
    against the fine solution there is of the size the paper describes for four to five
    iterations (O(1e-4)); this part is qualitative, the paper's u0 is not printed.
    """
    n = 63
    x = np.arange(1, n + 1) / (n + 1)
    u0 = 0.5 * np.sin(np.pi * x) + 0.2 * np.sin(3 * np.pi * x)
    p = o.Params(n=n, eps=0.0725, T=1.0, N=20, J=200, fine="nl", coarse="lin1", tol=1e-3)
    Uf = o.fine_solution(p, u0)
    r = o.parareal(p, u0, Uf)
    assert r.converged and r.iterations < p.N
    assert r.inc[-1] < 1e-3 and np.all(r.inc[:-1] >= 1e-3)
    assert r.err_l2[r.iterations] < 1e-3
    assert np.all(np.diff(r.err_l2[:5]) < 0)


# ------------------------------------------------------------- error norms (Section 4)
#
# The error and increment norms are pinned by discrete sine orthogonality, not by restating
# them: for 1 <= q <= n, sum_{j=1..n} sin^2(q pi j/(n+1)) = (n+1)/2, so the L2_h norm
# (h sum e^2)^(1/2) of c sin(q pi x) is |c|/sqrt(2) for every n. A wrong power of h, a missing
# square root or a sum over the wrong slices gives another value (one that depends on n).


@pytest.mark.parametrize("n", [7, 31, 64])
def test_error_norms_of_planted_sine_errors(n):
    """Uf = U^0 + c_s sin(q pi x): err_l2[0] = max_s |c_s|/sqrt(2), err_max[0] = max_s |c_s| max_j |sin|."""
    eps, T, N, J, pm, q = 0.0725, 1.0, 6, 20, 2, 5 if n > 5 else 1
    p = o.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1", frozen=True, max_iters=0)
    u0 = sine_mode(n, pm)
    a = frozen_parareal_closed_form(n, pm, eps, T, N, J, 0)  # U_s^0 = a^s u0 (Lemma 3.1)
    c = np.array([1e-3 * (s + 1) * (-1) ** s for s in range(N + 1)])
    Uf = a[:, None] * u0[None, :] + c[:, None] * sine_mode(n, q)[None, :]
    r = o.parareal(p, u0, Uf)
    assert r.iterations == 0
    want_l2 = np.max(np.abs(c)) / math.sqrt(2.0)
    want_mx = np.max(np.abs(c)) * np.max(np.abs(sine_mode(n, q)))
    # U^0 differs from the closed form by the coarse solves' rounding (~1e-13)
    assert abs(r.err_l2[0] - want_l2) <= 1e-12
    assert abs(r.err_max[0] - want_mx) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 4])
def test_error_and_increment_norms_follow_closed_form_iterates(k):
    """Frozen PA-I on one sine mode: U_s^k = c_s^k sin(p pi x) (Lemma 3.4) and the fine solution
    b^s sin(p pi x), so err_l2[k] = max_s |c_s^k - b^s| / sqrt(2) and
    inc[k-1] = max_s |c_s^k - c_s^(k-1)| max_j |sin(p pi x_j)|."""
    n, eps, T, N, J, pm = 31, 0.0725, 1.0, 8, 20, 3
    p = o.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1", frozen=True, max_iters=k)
    u0 = sine_mode(n, pm)
    y = mu(n, pm)
    dt = T / N / J
    b = ((1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)) ** J
    fine_coef = np.array([b ** s for s in range(N + 1)])
    Uf = fine_coef[:, None] * u0[None, :]
    r = o.parareal(p, u0, Uf)
    smax = np.max(np.abs(u0))
    for kk in range(k + 1):
        ck = frozen_parareal_closed_form(n, pm, eps, T, N, J, kk)
        d = np.max(np.abs(ck - fine_coef))
        assert abs(r.err_l2[kk] - d / math.sqrt(2.0)) <= 1e-12, kk
        assert abs(r.err_max[kk] - d * smax) <= 1e-12, kk
        if kk >= 1:
            cprev = frozen_parareal_closed_form(n, pm, eps, T, N, J, kk - 1)
            dinc = np.max(np.abs(ck - cprev)) * smax
            assert abs(r.inc[kk - 1] - dinc) <= 1e-12, kk


def test_energy_closed_form_on_sine_mode():
    """Eq. 1.2 on u = A sin(p pi x): h sum sin^2 = 1/2, h sum sin^4 = 3/8 (2p not a multiple of
    n+1) and u^T(-D_h)u = mu_p sum u^2, so E = (3A^4/8 - A^2 + n h)/4 + eps^2 mu_p A^2 / 4."""
    n, eps, pm, A = 40, 0.2, 3, 0.7
    h = 1.0 / (n + 1)
    want = (3 * A ** 4 / 8 - A ** 2 + n * h) / 4 + eps ** 2 * mu(n, pm) * A ** 2 / 4
    assert abs(o.energy(A * sine_mode(n, pm), eps) - want) <= 1e-12 * abs(want)

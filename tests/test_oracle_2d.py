"""Pins of the two-dimensional CPU oracle against facts the paper and mathematics fix."""
import math

import numpy as np
import pytest

import ch_inputs
from oracle import oracle1d as o1
from oracle import oracle2d as o2


def mu(n, p):
    h = 1.0 / (n + 1)
    return -(2.0 / h ** 2) * (math.cos(p * math.pi / (n + 1)) - 1.0)


def mode2(n, p, q):
    x = np.arange(1, n + 1) / (n + 1)
    return np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x)).reshape(-1)  # row y, column x


def test_dh_2d_eigenvalues_are_sums_of_1d_eigenvalues():
    n = 9
    D = o2.dh_matrix(n).toarray()
    ev = np.sort(np.linalg.eigvalsh(D))
    lam = np.sort([-(mu(n, p) + mu(n, q)) for p in range(1, n + 1) for q in range(1, n + 1)])
    assert np.max(np.abs(ev - lam) / np.abs(lam)) < 1e-12


def test_dh_2d_matches_kronecker_of_pinned_1d_operator():
    n = 6
    d1 = np.stack([o1.dh_apply(np.eye(n)[:, j]) for j in range(n)], axis=1)  # the pinned 1D oracle
    ref = np.kron(np.eye(n), d1) + np.kron(d1, np.eye(n))
    assert np.array_equal(o2.dh_matrix(n).toarray(), ref)


def test_mode_is_eigenvector_with_x_fastest_layout():
    n = 12
    v = mode2(n, 2, 5)
    lam = -(mu(n, 2) + mu(n, 5))
    assert np.allclose(o2.dh_apply(v, n), lam * v, atol=1e-9 * abs(lam))


@pytest.mark.parametrize("scheme", ["lin1", "lin2"])
def test_linear_steps_match_dense_brute_force(scheme):
    n, eps, dt = 5, 0.1, 1e-3
    u = ch_inputs.initial_condition(2, n, 3, amp=0.8)
    d1 = np.stack([o1.dh_apply(np.eye(n)[:, j]) for j in range(n)], axis=1)
    D = np.kron(np.eye(n), d1) + np.kron(d1, np.eye(n))
    I = np.eye(n * n)
    if scheme == "lin1":
        ref = np.linalg.solve(I - dt * D @ np.diag(u ** 2) + eps ** 2 * dt * D @ D, u - dt * D @ u)
    else:
        ref = np.linalg.solve(I - 2 * dt * D + eps ** 2 * dt * D @ D, u + dt * D @ u ** 3 - 3 * dt * D @ u)
    out, _ = o2.step(o2.Params(n=n, eps=eps, T=1, N=1, J=1), scheme, dt, u)
    assert np.max(np.abs(out - ref)) < 1e-12


def test_newton_step_is_root_of_eq_3_17():
    n, eps, dt = 7, 0.1, 5e-3
    u = ch_inputs.initial_condition(2, n, 4, amp=0.9)
    y, m = o2.step(o2.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13), "nl", dt, u)
    D = o2.dh_matrix(n).toarray()
    H = y + eps ** 2 * dt * D @ D @ y - dt * D @ y ** 3 - (u - dt * D @ u)
    assert np.max(np.abs(H)) < 1e-11
    assert 2 <= m <= 8


def _dh2_extended(v, n):
    """2D D_h (five-point, zero Dirichlet values, row-major) in numpy's extended precision."""
    w = np.zeros((n + 2, n + 2), dtype=np.longdouble)
    w[1:-1, 1:-1] = v.reshape(n, n)
    out = w[:-2, 1:-1] + w[2:, 1:-1] + w[1:-1, :-2] + w[1:-1, 2:] - 4 * w[1:-1, 1:-1]
    return (out * np.longdouble((n + 1) ** 2)).reshape(-1)


@pytest.mark.parametrize("n,eps,dt,tol", [
    (63, 0.01, 2.0 / (64 * 100), 1e-12),   # the 512 x 512 workload's eps and fine step, coarser grid
    (127, 0.01, 2.0 / (64 * 100), 1e-12),
    (63, 0.05, 1e-3, 1e-10),
])
def test_newton_stops_at_the_root_within_the_rounding_floor_2d(n, eps, dt, tol):
    """2D counterpart of the 1D pin: wherever Newton stops, one correction with the residual of
    Eq. 3.17 evaluated in extended precision moves the step by at most
    max(tol, u * 64 eps^2 dt / h^4 * max|Y|)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("no extended precision on this platform")
    u = ch_inputs.initial_condition(2, n, 5, amp=0.9)
    y, _ = o2.step(o2.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=tol), "nl", dt, u)
    Y, U, dtl = y.astype(np.longdouble), u.astype(np.longdouble), np.longdouble(dt)
    H = (Y + np.longdouble(eps) ** 2 * dtl * _dh2_extended(_dh2_extended(Y, n), n) - dtl * _dh2_extended(Y ** 3, n)
         - (U - dtl * _dh2_extended(U, n)))
    D = o2.dh_matrix(n)
    Jac = sp.identity(n * n, format="csc") + eps ** 2 * dt * (D @ D) - 3 * dt * (D @ sp.diags(y ** 2))
    dist = np.max(np.abs(spl.spsolve(Jac.tocsc(), H.astype(np.float64))))
    floor = np.finfo(np.float64).eps * 64 * eps ** 2 * dt * (n + 1) ** 4 * np.max(np.abs(y))
    assert dist <= max(tol, floor), (dist, tol, floor)


@pytest.mark.parametrize("scheme,i", [("lin1", 1), ("lin2", 2), ("nl", 1)])
def test_frozen_step_factor_lemma_3_1(scheme, i):
    n, eps, dt = 15, 0.07, 2e-3
    p = o2.Params(n=n, eps=eps, T=1, N=1, J=1, frozen=True)
    for (a, b) in ((1, 1), (3, 7), (15, 2)):
        v = mode2(n, a, b)
        out, _ = o2.step(p, scheme, dt, v)
        y = mu(n, a) + mu(n, b)
        g = (1 + i * dt * y) / (1 + i * dt * y + eps ** 2 * dt * y ** 2)
        assert np.max(np.abs(out - g * v)) < 1e-12


def mms_forcing_2d(eps):
    """u = e^{-t} sin(pi x) sin(pi y) solves u_t + eps^2 D^2 u = D(u^3 - u) + g with this g."""
    pi2 = np.pi ** 2
    return [(-1 + 4 * eps ** 2 * pi2 ** 2 - 2 * pi2, -1.0, 1, 1),
            (18 * pi2 / 16, -3.0, 1, 1), (-30 * pi2 / 16, -3.0, 1, 3), (-30 * pi2 / 16, -3.0, 3, 1),
            (18 * pi2 / 16, -3.0, 3, 3)]


def mms_error_2d(scheme, n, nsteps, T, eps=0.1):
    u0 = mode2(n, 1, 1)
    p = o2.Params(n=n, eps=eps, T=T, N=1, J=nsteps, newton_tol=1e-13)
    uT = o2.propagate(p, scheme, T / nsteps, nsteps, u0, forcing=mms_forcing_2d(eps))
    return np.max(np.abs(uT - math.exp(-T) * u0))


@pytest.mark.parametrize("scheme", ["nl", "lin1"])
def test_mms_2d_first_order_in_time(scheme):
    """Temporal error on a fixed grid, measured against a 32x finer step (the spatial O(h^2)
    error of the manufactured solution is common to both and cancels)."""
    n, T, eps = 31, 0.1, 0.1
    u0 = mode2(n, 1, 1)
    p = o2.Params(n=n, eps=eps, T=T, N=1, J=1, newton_tol=1e-13)
    f = mms_forcing_2d(eps)
    ref = o2.propagate(p, scheme, T / 640, 640, u0, forcing=f)
    errs = [np.max(np.abs(o2.propagate(p, scheme, T / m, m, u0, forcing=f) - ref)) for m in (10, 20, 40)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.75 < r1 < 2.4 and 1.75 < r2 < 2.4, errs


@pytest.mark.parametrize("scheme", ["nl"])
def test_mms_2d_second_order_in_space(scheme):
    errs = [mms_error_2d(scheme, n, 400, 0.01) for n in (7, 15, 31)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.4 < r1 < 4.8 and 3.4 < r2 < 4.6, errs


def test_eyre_energy_decay_2d():
    n, eps = 15, 0.08
    u = ch_inputs.initial_condition(2, n, 8, amp=0.5)
    p = o2.Params(n=n, eps=eps, T=1, N=1, J=1, newton_tol=1e-13)
    E = [o2.energy(u, n, eps)]
    for dt in [1e-3] * 4 + [5e-2] * 3:
        u, _ = o2.step(p, "nl", dt, u)
        E.append(o2.energy(u, n, eps))
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))


def test_frozen_parareal_closed_form_2d():
    n, eps, T, N, J = 15, 0.0725, 1.0, 6, 10
    a_, b_ = 2, 3
    u0 = mode2(n, a_, b_)
    y = mu(n, a_) + mu(n, b_)
    dT, dt = T / N, T / N / J
    a = (1 + dT * y) / (1 + dT * y + eps ** 2 * dT * y ** 2)
    b = ((1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)) ** J
    for k in (1, 3):
        r = o2.parareal(o2.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1", frozen=True), u0,
                        max_iters=k)
        coef = np.array([sum(math.comb(s, j) * (b - a) ** j * a ** (s - j) for j in range(min(k, s) + 1))
                         for s in range(N + 1)])
        assert np.max(np.abs(r.U - coef[:, None] * u0[None, :])) < 1e-12


def test_parareal_2d_finite_step_exactness():
    n, N = 9, 4
    u0 = ch_inputs.initial_condition(2, n, 1, amp=0.3)
    p = o2.Params(n=n, eps=0.1, T=0.02, N=N, J=5, fine="nl", coarse="lin1")
    Uf = o2.fine_solution(p, u0)
    for k in range(N + 1):
        r = o2.parareal(p, u0, Uf, max_iters=k)
        assert np.array_equal(r.U[: k + 1], Uf[: k + 1])
    assert r.err_max[-1] == 0.0


def test_2d_parareal_agrees_with_1d_oracle_on_separable_frozen_data():
    """Frozen LIN1 on u0 = sin(p pi x) sin(q pi y) equals the 1D oracle's per-mode factor product:
    both reduce to scalar recurrences with the same amplification (Lemma 3.1)."""
    n, eps, dt = 11, 0.05, 1e-3
    u0 = mode2(n, 4, 1)
    out = o2.propagate(o2.Params(n=n, eps=eps, T=1, N=1, J=1, frozen=True), "lin1", dt, 3, u0)
    y = mu(n, 4) + mu(n, 1)
    g = (1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)
    assert np.max(np.abs(out - g ** 3 * u0)) < 1e-13


def test_sine_transform_diagonalises_dh_and_is_involutory():
    n = 15
    x = ch_inputs.initial_condition(2, n, 12, amp=1.0).reshape(n, n)
    X = o2.sine_transform(x)
    assert np.allclose(o2.sine_transform(X), x, atol=1e-13)
    # D_h x in sine space is -(mu_p + mu_q) X (eigenvalues below Eq. 3.2)
    lam = np.array([[-(mu(n, q) + mu(n, p)) for p in range(1, n + 1)] for q in range(1, n + 1)])
    DX = o2.sine_transform(o2.dh_apply(x.reshape(-1), n).reshape(n, n))
    assert np.allclose(DX, lam * X, atol=1e-9 * np.abs(lam).max())
    # a single sine mode maps to a single coefficient
    v = mode2(n, 3, 5).reshape(n, n)
    V = o2.sine_transform(v)
    assert abs(V[4, 2]) > 1 and np.sum(np.abs(V) > 1e-9) == 1


# ------------------------------------------------------------- error norms (Section 4)
#
# Pinned by discrete sine orthogonality: h^2 sum_{i,j} sin^2(p pi x_i) sin^2(q pi y_j) = 1/4 for
# 1 <= p, q <= n, so the L2_h norm (h^2 sum e^2)^(1/2) of c sin(p pi x) sin(q pi y) is |c|/2.


@pytest.mark.parametrize("n", [7, 15])
def test_error_norms_of_planted_sine_errors_2d(n):
    eps, T, N, J = 0.0725, 1.0, 4, 5
    p = o2.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1", frozen=True)
    u0 = mode2(n, 2, 1)
    y = mu(n, 2) + mu(n, 1)
    dT = T / N
    a = (1 + dT * y) / (1 + dT * y + eps ** 2 * dT * y ** 2)
    c = np.array([2e-3 * (s + 1) * (-1) ** s for s in range(N + 1)])
    e = mode2(n, 3, 4)
    Uf = np.array([a ** s for s in range(N + 1)])[:, None] * u0[None, :] + c[:, None] * e[None, :]
    r = o2.parareal(p, u0, Uf, max_iters=0)
    want_l2 = np.max(np.abs(c)) / 2.0
    want_mx = np.max(np.abs(c)) * np.max(np.abs(e))
    assert abs(r.err_l2[0] - want_l2) <= 1e-12
    assert abs(r.err_max[0] - want_mx) <= 1e-12


def test_error_norms_follow_closed_form_iterates_2d():
    n, eps, T, N, J = 15, 0.0725, 1.0, 6, 10
    u0 = mode2(n, 2, 3)
    y = mu(n, 2) + mu(n, 3)
    dT, dt = T / N, T / N / J
    a = (1 + dT * y) / (1 + dT * y + eps ** 2 * dT * y ** 2)
    b = ((1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)) ** J
    fine_coef = np.array([b ** s for s in range(N + 1)])
    Uf = fine_coef[:, None] * u0[None, :]
    k = 3
    r = o2.parareal(o2.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1", frozen=True), u0, Uf,
                    max_iters=k)

    def coef(kk):
        return np.array([sum(math.comb(s, j) * (b - a) ** j * a ** (s - j) for j in range(min(kk, s) + 1))
                         for s in range(N + 1)])

    smax = np.max(np.abs(u0))
    for kk in range(k + 1):
        d = np.max(np.abs(coef(kk) - fine_coef))
        assert abs(r.err_l2[kk] - d / 2.0) <= 1e-12
        assert abs(r.err_max[kk] - d * smax) <= 1e-12
        if kk >= 1:
            dinc = np.max(np.abs(coef(kk) - coef(kk - 1))) * smax
            assert abs(r.inc[kk - 1] - dinc) <= 1e-12


def test_energy_closed_form_on_sine_mode_2d():
    """Eq. 1.2 on u = A sin(p pi x) sin(q pi y): h^2 sum u^2 = A^2/4, h^2 sum u^4 = 9A^4/64 (2p, 2q
    not multiples of n+1) and u^T(-D_h)u = (mu_p + mu_q) sum u^2, so
    E = (9A^4/64 - A^2/2 + (n h)^2)/4 + eps^2 (mu_p + mu_q) A^2 / 8."""
    n, eps, A = 15, 0.1, 0.8
    h = 1.0 / (n + 1)
    want = (9 * A ** 4 / 64 - A ** 2 / 2 + (n * h) ** 2) / 4 + eps ** 2 * (mu(n, 3) + mu(n, 2)) * A ** 2 / 8
    assert abs(o2.energy(A * mode2(n, 3, 2), n, eps) - want) <= 1e-12 * abs(want)


# ---------------------------------------------------- CG solver of the oracle (large grids)


@pytest.mark.parametrize("scheme,frozen", [("lin1", False), ("lin1", True), ("lin2", False), ("nl", False),
                                           ("nl", True)])
@pytest.mark.parametrize("n", [15, 31])
def test_pcg_solver_matches_sparse_direct(scheme, frozen, n):
    """The CG path (library CG on A^{-1} J, sine-transform preconditioner, refinement) reaches the
    sparse-LU step to rounding: a wrong operator in it (a sign, a missing eps^2 dt A term, a
    transposed transform) moves the result by far more."""
    u = ch_inputs.initial_condition(2, n, 21, kind="normal", amp=0.6)
    for dt in (1e-4, 2e-2):
        kw = dict(n=n, eps=0.03, T=1, N=1, J=1, frozen=frozen, newton_tol=1e-12)
        a, ma = o2.step(o2.Params(**kw), scheme, dt, u)
        b, mb = o2.step(o2.Params(**kw, solver="pcg"), scheme, dt, u)
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(a))), (dt, np.max(np.abs(a - b)))
        assert abs(ma - mb) <= 1

"""GPU parity of the Neumann-Neumann fine solver (Section 4.6, 1D) against the NN oracle: the
sequential fine solution, Parareal iterates with it as F, finite-step exactness, and the
iteration counts on a case whose convergence is known exactly."""
import numpy as np
import pytest

import ch_inputs
from oracle import nn1d
from oracle import oracle1d as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def nn_reference(n, eps, T, N, J, u0, N0, theta, tol, frozen=False):
    dt = T / N / J
    U = [np.asarray(u0, dtype=np.float64)]
    for _ in range(N):
        u, _ = nn1d.nn_propagate(n, eps, dt, J, U[-1], N0, theta, tol, frozen=frozen)
        U.append(u)
    return np.stack(U)


@pytest.mark.parametrize("n,N0", [(63, 8), (127, 8), (95, 4), (31, 1)])
def test_nn_reference_matches_oracle(gpu_lib, n, N0):
    """Tight interface tolerance: both sides converge to the global step, to rounding."""
    ch = gpu_lib
    eps, T, N, J = 0.0725, 0.02, 3, 4
    u0 = ch_inputs.initial_condition(1, n, 30, amp=0.3)
    cfg = ch.Config(n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", precision=0, max_iters=1)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_fine_nn(N0, theta=0.25, tol=1e-13, max_iter=400)
        pr.set_initial(0, u0)
        pr.compute_reference()
        Ug = pr.get_reference(0)
    Uo = nn_reference(n, eps, T, N, J, u0, N0, 0.25, 1e-13)
    assert np.max(np.abs(Ug - Uo)) <= 1e-11 * max(1.0, np.max(np.abs(Uo)))
    # and the monolithic scheme Eq. 2.4
    ref = o.fine_solution(o.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1"), u0)
    assert np.max(np.abs(Ug - ref)) <= 1e-10


def test_nn_reference_at_the_papers_tolerance(gpu_lib):
    """The paper's setting (8 subdomains, theta = 1/4, 1e-10 on the interface updates): GPU and
    oracle stop at the same iterations here, so they agree to rounding."""
    ch = gpu_lib
    n, eps, T, N, J = 127, 0.0725, 0.05, 4, 20
    u0 = ch_inputs.initial_condition(1, n, 0, amp=0.1)
    cfg = ch.Config(n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", precision=0, max_iters=1)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_fine_nn(8)
        pr.set_initial(0, u0)
        pr.compute_reference()
        Ug = pr.get_reference(0)
    Uo = nn_reference(n, eps, T, N, J, u0, 8, 0.25, 1e-10)
    assert np.max(np.abs(Ug - Uo)) <= 1e-9


def py_parareal(n, eps, T, N, J, u0, N0, theta, tol, kmax):
    """Eq. 2.2 with F the NN solver and G one step of Eq. 2.4 of dT (oracle), correction
    F(U_n^k) + (G(U_n^{k+1}) - G(U_n^k))."""
    p = o.Params(n=n, eps=eps, T=T, N=N, J=J, fine="lin1", coarse="lin1")
    dT = T / N

    def G(u):
        return o.propagate(p, "lin1", dT, 1, u)

    def F(u):
        return nn1d.nn_propagate(n, eps, dT / J, J, u, N0, theta, tol)[0]

    U = [np.asarray(u0, dtype=np.float64)]
    Gold = []
    for s in range(N):
        g = G(U[s])
        Gold.append(g)
        U.append(g)
    for k in range(kmax):
        Fk = {s: F(U[s]) for s in range(k, N)}
        newU = U[:k + 1]
        for s in range(k, N):
            g = G(newU[s])
            newU.append(Fk[s] + (g - Gold[s]))
            Gold[s] = g
        U = newU
    return np.stack(U)


def test_parareal_with_nn_fine_solver_matches_oracle_and_is_exact_at_k_equal_n(gpu_lib):
    ch = gpu_lib
    n, eps, T, N, J = 63, 0.0725, 0.02, 4, 5
    u0 = ch_inputs.initial_condition(1, n, 31, amp=0.3)
    for k in (1, 2):
        cfg = ch.Config(n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", precision=0, max_iters=k)
        with ch.Parareal(cfg, batch=1) as pr:
            pr.set_fine_nn(8, tol=1e-13, max_iter=400)
            pr.set_initial(0, u0)
            pr.run()
            U = pr.get_slices(0)
            st = pr.stats(0)
        ref = py_parareal(n, eps, T, N, J, u0, 8, 0.25, 1e-13, k)
        assert st["iterations"] == k
        assert np.max(np.abs(U - ref)) <= 1e-11
        assert st["newton_total"] > 0
    cfg = ch.Config(n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", precision=0, max_iters=N)
    with ch.Parareal(cfg, batch=2) as pr:
        pr.set_fine_nn(8)
        pr.set_initial_batch(np.stack([u0, 0.5 * u0]))
        pr.compute_reference()
        pr.run()
        for b in range(2):
            assert np.array_equal(pr.get_slices(b), pr.get_reference(b))


def test_two_mirror_symmetric_subdomains_take_two_iterations_per_step(gpu_lib):
    """Symmetric data stays symmetric under the scheme, so with two subdomains and theta = 1/4
    every step converges after one update (the second iteration confirms it)."""
    ch = gpu_lib
    n, eps, T, N, J = 63, 0.0725, 0.01, 2, 3
    half = ch_inputs.initial_condition(1, 32, 9, amp=0.5)
    u0 = np.concatenate([half[:31], [0.3], half[:31][::-1]])
    cfg = ch.Config(n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", precision=0, max_iters=1)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_fine_nn(2, theta=0.25, tol=1e-12)
        pr.set_initial(0, u0)
        pr.run()
        st = pr.stats(0)
    assert st["newton_max"] == 2
    assert st["newton_total"] == 2 * J * N


def test_set_fine_nn_rejects_bad_arguments(gpu_lib):
    ch = gpu_lib
    cfg = ch.Config(n=63, eps=0.05, T=0.01, n_slices=2, fine_steps=2, variant="PA-I", precision=0)
    with ch.Parareal(cfg, batch=1) as pr:
        for args in ((5,), (8, 0.0), (8, 1.5), (8, 0.25, 0.0), (8, 0.25, 1e-10, 0), (33,), (64,)):
            with pytest.raises(ch.ChError):
                pr.set_fine_nn(*args)
    cfg = ch.Config(n=63, eps=0.05, T=0.01, n_slices=2, fine_steps=2, variant="NPA-I", precision=0)
    with ch.Parareal(cfg, batch=1) as pr:
        with pytest.raises(ch.ChError):
            pr.set_fine_nn(8)

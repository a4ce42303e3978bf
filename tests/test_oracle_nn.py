"""Pins of the Neumann-Neumann oracle (oracle/nn1d.py), CPU only.

The NN iteration's fixed point is the global step of Eq. 2.4, which the C oracle computes by
banded elimination with no subdomains at all: a wrong interface split, residual sign, Neumann
data or update factor either breaks that equality or the one-update convergence that the
theory gives for two mirror-symmetric subdomains with theta = 1/4.
"""
import numpy as np
import pytest

import ch_inputs
from oracle import nn1d
from oracle import oracle1d as o


def test_local_matrices_sum_to_the_global_matrix():
    n, eps, dt, N0 = 31, 0.07, 1e-3, 4
    m = (n + 1) // N0
    un = ch_inputs.initial_condition(1, n, 3, amp=0.6)
    c2 = un * un
    A = nn1d.global_matrix(n, eps, dt, c2)
    S = np.zeros_like(A)
    for i in range(N0):
        a = i * m - 1 if i > 0 else 0
        b = (i + 1) * m - 1 if i < N0 - 1 else n - 1
        L = nn1d.local_matrix(n, eps, dt, c2, a, b, i > 0, i < N0 - 1)
        S[2 * a:2 * b + 2, 2 * a:2 * b + 2] += L
    assert np.array_equal(S, A) or np.max(np.abs(S - A)) <= 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("frozen", [False, True])
@pytest.mark.parametrize("n,N0", [(63, 8), (127, 8), (63, 2), (95, 3)])
def test_converged_step_is_the_banded_lin1_step(n, N0, frozen):
    eps, dt = 0.0725, 2e-5
    un = ch_inputs.initial_condition(1, n, 5, amp=0.4)
    u, it = nn1d.nn_step(n, eps, dt, un, N0, tol=1e-14, max_iter=400, frozen=frozen)
    ref, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1, frozen=frozen), "lin1", dt, un)
    assert 1 <= it < 400
    assert np.max(np.abs(u - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_single_subdomain_is_the_direct_solve():
    n, eps, dt = 47, 0.05, 1e-4
    un = ch_inputs.initial_condition(1, n, 8, amp=0.5)
    u, it = nn1d.nn_step(n, eps, dt, un, 1)
    ref, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1), "lin1", dt, un)
    assert it == 0
    assert np.max(np.abs(u - ref)) <= 1e-13


def test_two_mirror_symmetric_subdomains_converge_after_one_update():
    """S_1 = S_2 (mirror images), so theta (S_1^-1 + S_2^-1) = S^-1 at theta = 1/4: the first update
    gives the exact interface values and the second is at the rounding level."""
    n, eps, dt = 63, 0.0725, 5e-4
    half = ch_inputs.initial_condition(1, 32, 9, amp=0.5)
    un = np.concatenate([half[:31], [0.3], half[:31][::-1]])  # symmetric about the centre node 31
    assert np.array_equal(un, un[::-1])
    u, it = nn1d.nn_step(n, eps, dt, un, 2, theta=0.25, tol=1e-12)
    ref, _ = o.step(o.Params(n=n, eps=eps, T=1, N=1, J=1), "lin1", dt, un)
    assert it == 2
    assert np.max(np.abs(u - ref)) <= 1e-12


def test_propagation_and_iteration_counts():
    """Several steps (the fine propagator of a slice): equal to the banded propagation; the
    paper's setting (8 subdomains, theta = 1/4, tolerance 1e-10) needs few iterations per step."""
    n, eps, dt, steps = 127, 0.0725, 1e-4, 5
    un = ch_inputs.initial_condition(1, n, 12, amp=0.3)
    u, total = nn1d.nn_propagate(n, eps, dt, steps, un, 8, theta=0.25, tol=1e-10)
    ref = o.propagate(o.Params(n=n, eps=eps, T=1, N=1, J=1), "lin1", dt, steps, un)
    assert total <= 40 * steps
    assert np.max(np.abs(u - ref)) <= 1e-8

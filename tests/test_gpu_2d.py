"""GPU parity of the two-dimensional path against the CPU oracle (sparse direct solves).

Tolerances follow the 1D reasoning: one FP64 step is determined to about
u (1 + 64 alpha + 8 beta max w), alpha = eps^2 dt / h^4, beta = c dt / h^2 (the 13-point D_h^2
has row sum 64/h^4); single steps allow 64 times that per step. The sine transform runs in
FP32 (radix-2 FFT of length 2(n+1)): 1e-5 of the largest coefficient.
"""
import math

import numpy as np
import pytest

import ch_inputs
from oracle import oracle2d as o2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_ROUND = 2.0 ** -53
FINE_OF = {"PA-I": "lin1", "PA-II": "lin2", "PA-III": "lin2", "NPA-I": "nl", "NPA-II": "nl"}
COARSE_OF = {"PA-I": "lin1", "PA-II": "lin2", "PA-III": "lin1", "NPA-I": "lin1", "NPA-II": "nl"}


def step_bound_2d(n, eps, dt, c=3.0, wmax=1.0):
    h = 1.0 / (n + 1)
    return U_ROUND * (1 + 64 * eps ** 2 * dt / h ** 4 + 8 * c * dt / h ** 2 * wmax)


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def mode2(n, p, q):
    x = np.arange(1, n + 1) / (n + 1)
    return np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x)).reshape(-1)


@pytest.mark.parametrize("n", [15, 31, 63, 127, 255, 511])
def test_sine_transform_matches_oracle(gpu_lib, n):
    """FP32 2D DST-I against the oracle's FP64 one, and its own inverse. At n = 255 and 511 each
    row's DST comes from an FFT of length n + 1 whose odd coefficients are running sums of FFT
    outputs: their rounding accumulates along the sum (FP32 emulation at n = 511: 7.8e-7 of the
    maximum per 2D transform, 3.1e-6 after two; at 255: 6.6e-7 and 1.5e-6), hence the looser
    bound there; the odd-extension FFT of the other sizes stays near 1e-7."""
    ch = gpu_lib
    tol = 3e-5 if n >= 255 else 1e-5
    x = np.stack([ch_inputs.initial_condition(2, n, 50 + b, kind="normal", amp=1.0).reshape(n, n)
                  for b in range(3)]).astype(np.float32)
    X = ch.sine_transform_2d(dev(x, torch.float32)).cpu().numpy()
    ref = o2.sine_transform(x.astype(np.float64))
    err = np.max(np.abs(X - ref)) / np.max(np.abs(ref))
    back = ch.sine_transform_2d(dev(X, torch.float32)).cpu().numpy()
    err_back = np.max(np.abs(back - x)) / np.max(np.abs(x))
    print(f"n={n}: transform {err:.2e}, round trip {err_back:.2e} of the maximum")
    assert err <= tol and err_back <= tol


@pytest.mark.parametrize("n", [15, 31, 63])
@pytest.mark.parametrize("scheme", ["lin1", "lin2", "nl"])
def test_propagate_2d_matches_oracle(gpu_lib, n, scheme):
    ch = gpu_lib
    h = 1.0 / (n + 1)
    eps = 0.05
    dt = min(1e-3, 2000.0 * h ** 4 / eps ** 2)
    nsteps, B = 3, 2
    u0 = np.stack([ch_inputs.initial_condition(2, n, 70 + b, amp=0.6) for b in range(B)])
    # Newton (and the refinement of the linear schemes) stops once its estimated remaining error
    # is below newton_tol: 1e-13 keeps that under the step bound the comparison uses
    cfg = ch.Config(dim=2, n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-13)
    out = ch.propagate(cfg, scheme, dt, nsteps, dev(u0)).cpu().numpy()
    p = o2.Params(n=n, eps=eps, T=1.0, N=1, J=1, newton_tol=1e-12)
    tol = 64 * step_bound_2d(n, eps, dt) * nsteps + 1e-13
    for b in range(B):
        ref = o2.propagate(p, scheme, dt, nsteps, u0[b])
        assert np.max(np.abs(out[b] - ref)) <= tol, (b, np.max(np.abs(out[b] - ref)), tol)


def test_frozen_2d_steps_match_lemma_3_1(gpu_lib):
    ch = gpu_lib
    n, eps, dt = 63, 0.07, 5e-4
    modes = [(1, 1), (5, 9), (60, 2)]
    u = np.stack([mode2(n, a, b) for a, b in modes])
    for scheme, i in (("lin1", 1), ("lin2", 2), ("nl", 1)):
        cfg = ch.Config(dim=2, n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, frozen=True)
        out = ch.propagate(cfg, scheme, dt, 1, dev(u)).cpu().numpy()
        for k, (a, b) in enumerate(modes):
            y = sum((2.0 * (n + 1) ** 2) * (1.0 - math.cos(m * math.pi / (n + 1))) for m in (a, b))
            g = (1 + i * dt * y) / (1 + i * dt * y + eps ** 2 * dt * y ** 2)
            assert np.max(np.abs(out[k] - g * u[k])) <= 64 * step_bound_2d(n, eps, dt, c=2.0), (scheme, a, b)


def oracle_params(cfg):
    return o2.Params(n=cfg.n, eps=cfg.eps, T=cfg.T, N=cfg.n_slices, J=cfg.fine_steps, coarse_steps=cfg.coarse_steps,
                     fine=FINE_OF[cfg.variant], coarse=COARSE_OF[cfg.variant], newton_tol=cfg.newton_tol,
                     frozen=cfg.frozen, tol=cfg.tol)


@pytest.mark.parametrize("variant", ["PA-I", "PA-II", "PA-III", "NPA-I", "NPA-II"])
def test_parareal_2d_matches_oracle_and_is_exact_at_k_equal_n(gpu_lib, variant):
    ch = gpu_lib
    n, N = 31, 4
    cfg = ch.Config(dim=2, n=n, eps=0.05, T=0.01, n_slices=N, fine_steps=4, variant=variant, newton_tol=1e-12)
    u0s = [ch_inputs.initial_condition(2, n, s, kind="normal", amp=0.05) for s in (1, 2)]
    pr = ch.Parareal(cfg, batch=2)
    for b, u in enumerate(u0s):
        pr.set_initial(b, u)
    pr.compute_reference()
    pr.run()
    tol = 64 * step_bound_2d(n, cfg.eps, cfg.T / N) * (N + cfg.fine_steps * N) + 1e-12
    for b, u0 in enumerate(u0s):
        U, Uref = pr.get_slices(b), pr.get_reference(b)
        assert np.array_equal(U, Uref)  # finite-step exactness (Theorem 3.2, remark closing Section 3)
        r = o2.parareal(oracle_params(cfg), u0)
        assert np.max(np.abs(U - r.U)) <= tol, (b, np.max(np.abs(U - r.U)), tol)
        st = pr.stats(b)
        assert st["iterations"] == N and st["err_max"][-1] == 0.0
    pr.close()


@pytest.mark.parametrize("k", [1, 2])
def test_parareal_2d_intermediate_iterates(gpu_lib, k):
    ch = gpu_lib
    n, N = 15, 5
    cfg = ch.Config(dim=2, n=n, eps=0.06, T=0.02, n_slices=N, fine_steps=3, variant="NPA-I", max_iters=k)
    u0 = ch_inputs.initial_condition(2, n, 9, kind="normal", amp=0.1)
    pr = ch.Parareal(cfg, batch=1)
    pr.set_initial(0, u0)
    pr.compute_reference()
    pr.run()
    U, Uref = pr.get_slices(0), pr.get_reference(0)
    assert np.array_equal(U[: k + 1], Uref[: k + 1])
    p = oracle_params(cfg)
    Uf = o2.fine_solution(p, u0)
    r = o2.parareal(p, u0, Uf, max_iters=k)
    tol = 64 * step_bound_2d(n, cfg.eps, cfg.T / N) * (2 * N + cfg.fine_steps * N) + 1e-12
    assert np.max(np.abs(U - r.U)) <= tol
    st = pr.stats(0)
    assert np.allclose(st["err_l2"], r.err_l2, rtol=1e-6, atol=tol)
    pr.close()


def test_frozen_parareal_2d_closed_form(gpu_lib):
    ch = gpu_lib
    n, eps, T, N, J = 31, 0.0725, 1.0, 6, 10
    a_, b_ = 2, 3
    u0 = mode2(n, a_, b_)
    y = sum((2.0 * (n + 1) ** 2) * (1.0 - math.cos(m * math.pi / (n + 1))) for m in (a_, b_))
    dT, dt = T / N, T / N / J
    a = (1 + dT * y) / (1 + dT * y + eps ** 2 * dT * y ** 2)
    b = ((1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)) ** J
    for k in (1, 3):
        cfg = ch.Config(dim=2, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", frozen=True, max_iters=k)
        pr = ch.Parareal(cfg, batch=1)
        pr.set_initial(0, u0)
        pr.run()
        coef = np.array([sum(math.comb(s, j) * (b - a) ** j * a ** (s - j) for j in range(min(k, s) + 1))
                         for s in range(N + 1)])
        assert np.max(np.abs(pr.get_slices(0) - coef[:, None] * u0[None, :])) <= 64 * step_bound_2d(n, eps, dT, c=1)
        pr.close()


def test_c3_grid_full_size_steps(gpu_lib):
    """The c3 configuration's grid and steps (256 x 256 grid: n = 255, eps = 0.01, coarse step
    dT = 0.5/32 with Eq. 2.4, fine step dt = dT/100 with Eq. 2.3, u0 = 0.05 N(0,1) seed 1): two
    coarse and two fine steps against the sparse-direct oracle."""
    ch = gpu_lib
    n, eps, T, N, J = 255, 0.01, 0.5, 32, 100
    u0 = ch_inputs.initial_condition(2, n, 1, kind="normal", amp=0.05)
    cfg = ch.Config(dim=2, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, newton_tol=1e-12)
    p = o2.Params(n=n, eps=eps, T=T, N=N, J=J, newton_tol=1e-12)
    dT, dt = T / N, T / N / J
    for scheme, step, c in (("lin1", dT, 1.0), ("nl", dt, 3.0)):
        out = ch.propagate(cfg, scheme, step, 2, dev(u0[None, :])).cpu().numpy()[0]
        ref = o2.propagate(p, scheme, step, 2, u0)
        tol = 64 * step_bound_2d(n, eps, step, c=c) * 2
        assert np.max(np.abs(out - ref)) <= tol, (scheme, np.max(np.abs(out - ref)), tol)


@pytest.fixture(params=["persistent", "cluster"])
def alt_path(request, monkeypatch):
    """Selects another execution of the 2D steps (read when a solver is created): the persistent
    cooperative kernel, or one thread-block cluster per unit."""
    monkeypatch.setenv("CH_2D_STEP", request.param)
    return request.param


@pytest.mark.parametrize("n", [15, 63, 255])
@pytest.mark.parametrize("scheme", ["lin1", "lin2", "nl"])
def test_other_paths_match_oracle(gpu_lib, alt_path, n, scheme):
    """The persistent and cluster executions (the default is one graph per step) against the
    oracle."""
    ch = gpu_lib
    h = 1.0 / (n + 1)
    eps = 0.05
    dt = min(1e-3, 2000.0 * h ** 4 / eps ** 2)
    nsteps, B = 2, 2
    u0 = np.stack([ch_inputs.initial_condition(2, n, 170 + b, amp=0.6) for b in range(B)])
    # Newton (and the refinement of the linear schemes) stops once its estimated remaining error
    # is below newton_tol: 1e-13 keeps that under the step bound the comparison uses
    cfg = ch.Config(dim=2, n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-13)
    out = ch.propagate(cfg, scheme, dt, nsteps, dev(u0)).cpu().numpy()
    p = o2.Params(n=n, eps=eps, T=1.0, N=1, J=1, newton_tol=1e-12)
    tol = 64 * step_bound_2d(n, eps, dt) * nsteps + 1e-13
    for b in range(B):
        ref = o2.propagate(p, scheme, dt, nsteps, u0[b])
        assert np.max(np.abs(out[b] - ref)) <= tol, (b, np.max(np.abs(out[b] - ref)), tol)


@pytest.mark.parametrize("n", [31, 255])
def test_persistent_and_graph_paths_agree(gpu_lib, monkeypatch, n):
    """Both executions run the same phase functions in the same order on the same data; compiled
    in different contexts they may contract multiply-adds differently, so they agree to the
    step's rounding floor. Each is deterministic."""
    ch = gpu_lib
    eps, dt, nsteps, B = 0.01, 1.5625e-4, 3, 4
    u0 = np.stack([ch_inputs.initial_condition(2, n, 300 + b, kind="normal", amp=0.05) for b in range(B)])
    cfg = ch.Config(dim=2, n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-12)
    g = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
    g2 = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
    monkeypatch.setenv("CH_2D_STEP", "persistent")
    a = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
    a2 = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
    assert np.array_equal(g, g2) and np.array_equal(a, a2)
    assert np.max(np.abs(a - g)) <= 64 * step_bound_2d(n, eps, dt) * nsteps


@pytest.mark.parametrize("n", [31, 255, 511])
def test_cluster_path_agrees_and_is_independent_of_cluster_size(gpu_lib, monkeypatch, n):
    """The cluster execution runs the graph path's phase functions per unit, so it agrees with it
    to the step's rounding floor; and each unit's arithmetic (row blocks, partial sums in block
    order) does not depend on how many blocks share the unit, so every cluster size gives the
    same bits."""
    ch = gpu_lib
    eps, dt, nsteps, B = 0.01, 1.5625e-4, 2, 3
    u0 = np.stack([ch_inputs.initial_condition(2, n, 330 + b, kind="normal", amp=0.05) for b in range(B)])
    cfg = ch.Config(dim=2, n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-12)
    g = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
    monkeypatch.setenv("CH_2D_STEP", "cluster")
    c = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
    assert np.max(np.abs(c - g)) <= 64 * step_bound_2d(n, eps, dt) * nsteps
    nb = (n + 15) // 16
    for size in (1, 2, 4, 8, 16):
        if nb % size:
            continue
        monkeypatch.setenv("CH_2D_CLUSTER", str(size))
        cs = ch.propagate(cfg, "nl", dt, nsteps, dev(u0)).cpu().numpy()
        assert np.array_equal(cs, c), size


@pytest.mark.parametrize("path", ["graph", "cluster"])
def test_parareal_2d_iterates_match_oracle_on_each_path(gpu_lib, monkeypatch, path):
    """Parareal (NPA-I) on a batch of two problems with the chosen 2D execution: the reference
    fine solution and two iterates follow the oracle."""
    ch = gpu_lib
    if path != "graph":
        monkeypatch.setenv("CH_2D_STEP", path)
    n, N, J, eps, T = 31, 4, 3, 0.05, 0.01
    cfg = ch.Config(dim=2, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="NPA-I", newton_tol=1e-12,
                    max_iters=2)
    u0s = [ch_inputs.initial_condition(2, n, 440 + b, kind="normal", amp=0.1) for b in range(2)]
    pr = ch.Parareal(cfg, batch=2)
    pr.set_initial_batch(np.stack(u0s))
    pr.compute_reference()
    pr.run()
    p = oracle_params(cfg)
    tol = 64 * step_bound_2d(n, eps, T / N) * (2 * N + J * N) + 1e-12
    for b in range(2):
        Uf = o2.fine_solution(p, u0s[b])
        r = o2.parareal(p, u0s[b], Uf, max_iters=2)
        assert np.max(np.abs(pr.get_reference(b) - Uf)) <= tol
        assert np.max(np.abs(pr.get_slices(b) - r.U)) <= tol
        assert pr.stats(b)["iterations"] == 2
    pr.close()


@pytest.mark.parametrize("path", ["graph", "cluster"])
def test_per_problem_eps_matches_oracle(gpu_lib, monkeypatch, path):
    """A batch whose problems have different eps (ch_parareal_set_eps): each problem's sequential
    fine solution and Parareal iterates follow the oracle run with its own eps."""
    ch = gpu_lib
    if path != "graph":
        monkeypatch.setenv("CH_2D_STEP", path)
    n, N, J = 31, 4, 3
    eps = [0.03, 0.05, 0.08]
    cfg = ch.Config(dim=2, n=n, eps=0.05, T=0.01, n_slices=N, fine_steps=J, variant="NPA-I", newton_tol=1e-12,
                    max_iters=2)
    u0s = [ch_inputs.initial_condition(2, n, 400 + b, kind="normal", amp=0.1) for b in range(3)]
    pr = ch.Parareal(cfg, batch=3)
    pr.set_initial_batch(np.stack(u0s))
    pr.set_eps(eps)
    pr.compute_reference()
    pr.run()
    for b in range(3):
        c = ch.Config(dim=2, n=n, eps=eps[b], T=0.01, n_slices=N, fine_steps=J, variant="NPA-I",
                      newton_tol=1e-12, max_iters=2)
        p = oracle_params(c)
        Uf = o2.fine_solution(p, u0s[b])
        r = o2.parareal(p, u0s[b], Uf, max_iters=2)
        tol = 64 * step_bound_2d(n, eps[b], 0.01 / N) * (2 * N + J * N) + 1e-12
        assert np.max(np.abs(pr.get_reference(b) - Uf)) <= tol
        assert np.max(np.abs(pr.get_slices(b) - r.U)) <= tol
    pr.close()


def test_ensemble_of_uneven_grids_matches_single_problem_runs(gpu_lib):
    """An ensemble groups its problems by grid size (one batched handle per size, run
    concurrently); each problem's iterates and reference equal those of its own single-problem
    handle (the 2D kernels treat every unit independently)."""
    ch = gpu_lib
    ns = [15, 31, 15, 31, 63]
    eps = [0.04, 0.06, 0.05, 0.03, 0.05]
    cfg = ch.Config(dim=2, n=15, eps=0.05, T=0.01, n_slices=4, fine_steps=3, variant="NPA-I", newton_tol=1e-12,
                    max_iters=3)
    u0s = [ch_inputs.initial_condition(2, n, 500 + i, kind="normal", amp=0.1) for i, n in enumerate(ns)]
    ens = ch.Ensemble(cfg, ns, eps)
    assert ens.groups == 3
    for i, u in enumerate(u0s):
        ens.set_initial(i, u)
    ens.compute_reference()
    ens.run()
    for i, (n, e) in enumerate(zip(ns, eps)):
        c = ch.Config(dim=2, n=n, eps=e, T=0.01, n_slices=4, fine_steps=3, variant="NPA-I", newton_tol=1e-12,
                      max_iters=3)
        pr = ch.Parareal(c, batch=1)
        pr.set_initial(0, u0s[i])
        pr.compute_reference()
        pr.run()
        assert np.array_equal(ens.get_slices(i), pr.get_slices(0)), i
        assert np.array_equal(ens.get_reference(i), pr.get_reference(0)), i
        assert ens.stats(i)["iterations"] == 3
        pr.close()
    ens.close()


def test_ensemble_over_the_c5_grid_sizes_matches_single_problem_runs(gpu_lib):
    """The ensemble's grid sizes of the uneven-grid configuration (64^2 .. 512^2: n = 63, 127, 255,
    511), each problem with its own eps: every problem's iterates equal those of its own
    single-problem handle bit for bit."""
    ch = gpu_lib
    ns = [63, 511, 127, 255, 63]
    eps = [0.01, 0.02, 0.05, 0.03, 0.04]
    kw = dict(dim=2, T=0.002, n_slices=4, fine_steps=2, variant="NPA-I", newton_tol=1e-12, max_iters=2)
    cfg = ch.Config(n=ns[0], eps=eps[0], **kw)
    u0s = [ch_inputs.initial_condition(2, n, 700 + i, kind="normal", amp=0.05) for i, n in enumerate(ns)]
    ens = ch.Ensemble(cfg, ns, eps)
    assert ens.groups == 4
    for i, u in enumerate(u0s):
        ens.set_initial(i, u)
    ens.run()
    for i, (n, e) in enumerate(zip(ns, eps)):
        pr = ch.Parareal(ch.Config(n=n, eps=e, **kw), batch=1)
        pr.set_initial(0, u0s[i])
        pr.run()
        assert np.array_equal(ens.get_slices(i), pr.get_slices(0)), (i, n)
        pr.close()
    ens.close()


@pytest.mark.parametrize("env", [None, "host", "persistent"])
def test_execution_is_reported(gpu_lib, monkeypatch, env):
    """The execution a handle's first run fixes: the one the environment names, else the tuner's
    choice between graphs and the persistent kernel; unknown before the first run."""
    ch = gpu_lib
    if env:
        monkeypatch.setenv("CH_2D_STEP", env)
    else:
        monkeypatch.delenv("CH_2D_STEP", raising=False)
    n = 31
    cfg = ch.Config(dim=2, n=n, eps=0.05, T=0.01, n_slices=2, fine_steps=2, variant="NPA-I", max_iters=1)
    with ch.Parareal(cfg, batch=1) as pr:
        assert pr.execution() == ""
        pr.set_initial(0, ch_inputs.initial_condition(2, n, 3, amp=0.3))
        pr.run()
        got = pr.execution()
    assert got == env if env else got in ("graphs", "persistent")


def test_unit_groups_do_not_change_results(gpu_lib, monkeypatch):
    """A batch of 16 or more units runs as up to four groups of step graphs on their own streams;
    the units are independent, so one group or four give the same bits."""
    ch = gpu_lib
    n, B = 31, 32
    u0 = np.stack([ch_inputs.initial_condition(2, n, 300 + b, amp=0.5) for b in range(B)])
    cfg = ch.Config(dim=2, n=n, eps=0.05, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-12)
    out = {}
    for groups in ("1", "4"):
        monkeypatch.setenv("CH_2D_GROUPS", groups)
        out[groups] = ch.propagate(cfg, "nl", 2e-4, 3, dev(u0)).cpu().numpy()
    assert np.array_equal(out["1"], out["4"])

"""GPU parity of the one-dimensional path against the CPU oracle, through the C ABI.

Tolerances. Two correct FP64 solvers of the implicit steps differ by the rounding of the
step matrix: its entries are up to 16 alpha with alpha = eps^2 dt / h^4 while the smooth
solution components see eigenvalues near 1, so one solve is accurate to about
u * (1 + 16 alpha + 4 beta max w), u = 2^-53, beta = c dt / h^2 (the same bound sets the
Newton rounding floor). Single-step tests allow 64 times that bound. Whole-run tests require
1e-11 or, where that is below what FP64 can resolve, four times the measured floor: the
difference between two correct FP64 oracles that run the same Newton iteration with
different rounding (Eq. 3.18 as printed, and the unsimplified step Y - J^-1 H(Y)). Spinodal
growth amplifies the per-step rounding, so at c2's size that floor is about 4e-7 after two
iterations.
"""
import math

import numpy as np
import pytest

import ch_inputs
from oracle import oracle1d as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_ROUND = 2.0 ** -53
FINE_OF = {"PA-I": "lin1", "PA-II": "lin2", "PA-III": "lin2", "NPA-I": "nl", "NPA-II": "nl"}
COARSE_OF = {"PA-I": "lin1", "PA-II": "lin2", "PA-III": "lin1", "NPA-I": "lin1", "NPA-II": "nl"}


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def step_bound(n, eps, dt, c=3.0, wmax=1.0):
    h = 1.0 / (n + 1)
    alpha = eps ** 2 * dt / h ** 4
    beta = c * dt / h ** 2
    return U_ROUND * (1 + 16 * alpha + 4 * beta * wmax)


def oracle_and_floor(p, u0, Ufine=None, residual_linear=False):
    """Oracle Parareal and its rounding floor (Eq. 3.18 form vs the unsimplified Newton form; with
    residual_linear, also the linear steps taken from their FP64 residual, as the GPU's FP32 solves
    refined in FP64 take them)."""
    r = o.parareal(p, u0, Ufine)
    if FINE_OF_SCHEME_NL(p) or residual_linear:
        q = o.Params(**{**p.__dict__, "newton_form": 1})
        floor = float(np.max(np.abs(o.parareal(q, u0).U - r.U)))
    else:
        floor = 0.0
    return r, max(1e-11, 4 * floor)


def FINE_OF_SCHEME_NL(p):
    return p.fine == "nl" or p.coarse == "nl"


def oracle_params(cfg, **kw):
    p = o.Params(n=cfg.n, eps=cfg.eps, T=cfg.T, N=cfg.n_slices, J=cfg.fine_steps, coarse_steps=cfg.coarse_steps,
                 fine=FINE_OF[cfg.variant], coarse=COARSE_OF[cfg.variant], newton_tol=cfg.newton_tol,
                 newton_max=cfg.newton_max, frozen=cfg.frozen, tol=cfg.tol,
                 max_iters=cfg.max_iters if cfg.max_iters > 0 else cfg.n_slices)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ----------------------------------------------------------------- single propagations


@pytest.mark.parametrize("n", [1, 2, 7, 64, 129, 300, 1000, 1024, 1500, 2048])
@pytest.mark.parametrize("scheme", ["lin1", "lin2", "nl"])
def test_propagate_matches_oracle(gpu_lib, n, scheme):
    ch = gpu_lib
    h = 1.0 / (n + 1)
    eps = 0.05
    dt = min(1e-3, 2000.0 * h ** 4 / eps ** 2)  # alpha <= 2000: a well-resolved step
    nsteps, B = 4, 3
    u0 = np.stack([ch_inputs.initial_condition(1, n, 100 + b, amp=0.6) for b in range(B)])
    tol = 64 * step_bound(n, eps, dt) * nsteps + 1e-14
    for precision in (0, 1):
        cfg = ch.Config(n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, newton_tol=1e-12, precision=precision)
        newton = torch.zeros(B, dtype=torch.int32, device="cuda")
        out = ch.propagate(cfg, scheme, dt, nsteps, dev(u0), newton=newton).cpu().numpy()
        p = o.Params(n=n, eps=eps, T=1.0, N=1, J=1, newton_tol=1e-12)
        for b in range(B):
            ref = o.propagate(p, scheme, dt, nsteps, u0[b])
            err = np.max(np.abs(out[b] - ref))
            assert err <= tol, (precision, b, err, tol)
        if scheme == "nl" or precision == 1:  # Newton, or refinement of the FP32 linear solves
            assert torch.all(newton >= nsteps).item() and torch.all(newton <= 12 * nsteps).item()
        else:
            assert torch.all(newton == 0).item()


def test_propagate_in_place_and_zero_state(gpu_lib):
    ch = gpu_lib
    n = 200
    cfg = ch.Config(n=n, eps=0.05, T=1.0, n_slices=1, fine_steps=1)
    u = torch.zeros(2, n, dtype=torch.float64, device="cuda")
    ch.propagate(cfg, "nl", 1e-4, 3, u, u_out=u)
    assert torch.count_nonzero(u).item() == 0
    u0 = ch_inputs.initial_condition(1, n, 9, amp=0.3)
    x = dev(np.stack([u0, u0]))
    y = ch.propagate(cfg, "lin1", 1e-4, 2, x.clone())
    ch.propagate(cfg, "lin1", 1e-4, 2, x, u_out=x)  # aliasing input and output
    assert torch.equal(x, y)


def test_frozen_steps_match_lemma_3_1_on_gpu(gpu_lib):
    """diag(u^2) = I: sine modes scale by g_i(mu_p) (Lemma 3.1), independently of the oracle."""
    ch = gpu_lib
    n, eps, dt = 255, 0.07, 2e-4
    x = np.arange(1, n + 1) / (n + 1)
    modes = [1, 17, 200]
    u = np.stack([np.sin(p * np.pi * x) for p in modes])
    for scheme, i in (("lin1", 1), ("lin2", 2), ("nl", 1)):
        cfg = ch.Config(n=n, eps=eps, T=1.0, n_slices=1, fine_steps=1, frozen=True, precision=0)
        out = ch.propagate(cfg, scheme, dt, 1, dev(u)).cpu().numpy()
        for k, p in enumerate(modes):
            y = (2.0 * (n + 1) ** 2) * (1.0 - math.cos(p * math.pi / (n + 1)))
            g = (1 + i * dt * y) / (1 + i * dt * y + eps ** 2 * dt * y ** 2)
            assert np.max(np.abs(out[k] - g * u[k])) < 64 * step_bound(n, eps, dt), (scheme, p)


# ------------------------------------------------------------------------- Parareal


def run_gpu(ch, cfg, u0s, reference=True):
    B = len(u0s)
    pr = ch.Parareal(cfg, batch=B)
    for b, u in enumerate(u0s):
        pr.set_initial(b, u)
    if reference:
        pr.compute_reference()
    status = pr.run()
    return pr, status


@pytest.mark.parametrize("precision", [0, 1])
def test_c1_linear_parareal_full_size_matches_oracle(gpu_lib, precision):
    """1D PA-I, M=128, eps=0.05, T=0.1, N=16, dt=1e-5, one coarse step, u0 = 0.1 U(-1,1) seed 0,
    stop at ||U^k - U^{k-1}||_inf < 1e-10; the fine steps as FP64 solves (precision 0) and as FP32
    solves refined against the FP64 residual (precision 1), both within the FP64 bound."""
    ch = gpu_lib
    cfg = ch.Config(n=128, eps=0.05, T=0.1, n_slices=16, fine_steps=625, variant="PA-I", tol=1e-10,
                    precision=precision)
    u0 = ch_inputs.initial_condition(1, 128, 0, amp=0.1)
    pr, status = run_gpu(ch, cfg, [u0])
    U = pr.get_slices(0)
    st = pr.stats(0)
    p = oracle_params(cfg)
    Uf = o.fine_solution(p, u0)
    r = o.parareal(p, u0, Uf)
    tol = 1e-11
    if precision == 1:
        # Each fine step is taken from its FP64 residual. The oracle's residual form of the same
        # steps differs from its direct solves by rounding only, amplified by the growth of the
        # unstable modes (about e^10 over T = 0.1 at eps = 0.05): that distance is the floor.
        Uf1 = o.fine_solution(oracle_params(cfg, newton_form=1), u0)
        floor = float(np.max(np.abs(Uf1 - Uf)))
        assert floor < 1e-10
        tol = max(tol, 4 * floor)
        assert np.max(np.abs(pr.get_reference(0) - Uf1)) <= tol
    assert np.max(np.abs(U - r.U)) <= tol
    assert np.max(np.abs(pr.get_reference(0) - Uf)) <= tol
    assert st["iterations"] == r.iterations
    assert st["converged"] == r.converged
    k = min(len(st["inc"]), len(r.inc))
    assert np.allclose(st["inc"][:k], r.inc[:k], rtol=1e-6, atol=tol)
    assert np.allclose(st["err_l2"], r.err_l2, rtol=1e-6, atol=tol)
    pr.close()


@pytest.mark.parametrize("variant", ["PA-I", "PA-II", "PA-III", "NPA-I", "NPA-II"])
@pytest.mark.parametrize("precision", [0, 1])
def test_all_variants_match_oracle_and_finite_step_exactness(gpu_lib, variant, precision):
    ch = gpu_lib
    n, N = 190, 6
    cfg = ch.Config(n=n, eps=0.06, T=0.02, n_slices=N, fine_steps=12, coarse_steps=2, variant=variant,
                    newton_tol=1e-12, precision=precision)
    u0s = [ch_inputs.initial_condition(1, n, s, amp=0.4) for s in (3, 4)]
    pr, status = run_gpu(ch, cfg, u0s)
    for b, u0 in enumerate(u0s):
        U = pr.get_slices(b)
        Uref = pr.get_reference(b)
        # Theorem 3.2 / remark closing Section 3: after N iterations the iterate is the fine solution
        assert np.array_equal(U, Uref)
        r, tol = oracle_and_floor(oracle_params(cfg), u0, residual_linear=precision == 1)
        assert np.max(np.abs(U - r.U)) <= tol, variant
        st = pr.stats(b)
        assert st["iterations"] == N
        assert st["err_max"][-1] == 0.0
    pr.close()


@pytest.mark.parametrize("k", [1, 2, 4])
def test_intermediate_iterates_match_oracle(gpu_lib, k):
    ch = gpu_lib
    n, N = 333, 8
    cfg = ch.Config(n=n, eps=0.05, T=0.05, n_slices=N, fine_steps=15, variant="NPA-I", max_iters=k,
                    newton_tol=1e-12, precision=1)
    u0 = ch_inputs.initial_condition(1, n, 21, amp=0.2)
    pr, _ = run_gpu(ch, cfg, [u0])
    U = pr.get_slices(0)
    Uref = pr.get_reference(0)
    assert np.array_equal(U[: k + 1], Uref[: k + 1])  # slices n <= k are exact (bitwise, same F)
    p = oracle_params(cfg)
    Uf = o.fine_solution(p, u0)
    r, tol = oracle_and_floor(p, u0, Uf)
    assert np.max(np.abs(U - r.U)) <= tol
    st = pr.stats(0)
    assert np.allclose(st["err_max"], r.err_max, rtol=1e-6, atol=tol)
    pr.close()


def test_frozen_parareal_matches_closed_form_on_gpu(gpu_lib):
    """Frozen model: U_s^k = sum_{j<=k} C(s,j)(b-a)^j a^{s-j} u0 per sine mode (Lemma 3.4)."""
    ch = gpu_lib
    n, eps, T, N, J, pm = 127, 0.0725, 1.0, 8, 20, 5
    x = np.arange(1, n + 1) / (n + 1)
    u0 = np.sin(pm * np.pi * x)
    y = (2.0 * (n + 1) ** 2) * (1.0 - math.cos(pm * math.pi / (n + 1)))
    dT, dt = T / N, T / N / J
    a = (1 + dT * y) / (1 + dT * y + eps ** 2 * dT * y ** 2)
    bb = ((1 + dt * y) / (1 + dt * y + eps ** 2 * dt * y ** 2)) ** J
    for k in (1, 3, 8):
        cfg = ch.Config(n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="PA-I", frozen=True, max_iters=k,
                        precision=0)
        pr, _ = run_gpu(ch, cfg, [u0], reference=False)
        U = pr.get_slices(0)
        coef = np.array([sum(math.comb(s, j) * (bb - a) ** j * a ** (s - j) for j in range(min(k, s) + 1))
                         for s in range(N + 1)])
        assert np.max(np.abs(U - coef[:, None] * u0[None, :])) < 64 * step_bound(n, eps, dt, c=1.0)
        pr.close()


def test_c2_full_size_sampled_problems(gpu_lib):
    """1D NPA-I, M=1024, eps=0.02, T=1, N=64, J=200, Newton tol 1e-12, batch 256, u0 = 0.1 U(-1,1)
    seeds 0..255, the launch configuration of the benchmark; two iterations; sampled problems are
    compared with the oracle within four times the oracle's own rounding floor."""
    ch = gpu_lib
    B = 256
    cfg = ch.Config(n=1024, eps=0.02, T=1.0, n_slices=64, fine_steps=200, variant="NPA-I", newton_tol=1e-12,
                    max_iters=2, precision=1)
    u0s = [ch_inputs.initial_condition(1, 1024, b, amp=0.1) for b in range(B)]
    pr, _ = run_gpu(ch, cfg, u0s, reference=False)
    p = oracle_params(cfg)
    for b in (0, 255):
        U = pr.get_slices(b)
        r, tol = oracle_and_floor(p, u0s[b])
        err = np.max(np.abs(U - r.U))
        assert err <= tol, (b, err, tol)
        # slice 1 after two iterations is exact: F(u0), far from the amplified tail
        assert np.max(np.abs(U[1] - r.U[1])) <= 64 * step_bound(1024, 0.02, 1.0 / 64 / 200) * 200
        assert pr.stats(b)["iterations"] == 2
    pr.close()


# ----------------------------------------------------------------- degenerate inputs


def test_degenerate_sizes_and_zero_initial_state(gpu_lib):
    ch = gpu_lib
    for n in (1, 2, 3):
        cfg = ch.Config(n=n, eps=0.1, T=0.01, n_slices=3, fine_steps=4, variant="NPA-I", precision=0)
        u0 = ch_inputs.initial_condition(1, n, 5, amp=0.5)
        pr, _ = run_gpu(ch, cfg, [u0])
        r = o.parareal(oracle_params(cfg), u0)
        assert np.max(np.abs(pr.get_slices(0) - r.U)) <= 1e-13
        pr.close()
    # one slice: Parareal is the fine solve after one iteration
    cfg = ch.Config(n=64, eps=0.05, T=0.01, n_slices=1, fine_steps=10, variant="NPA-I", tol=1e-10)
    u0 = ch_inputs.initial_condition(1, 64, 6, amp=0.5)
    pr, status = run_gpu(ch, cfg, [u0])
    assert np.array_equal(pr.get_slices(0), pr.get_reference(0))
    pr.close()
    # u0 = 0 is a fixed point of every scheme: the first increment is exactly zero
    cfg = ch.Config(n=100, eps=0.05, T=0.01, n_slices=4, fine_steps=5, variant="NPA-I", tol=1e-14)
    pr, status = run_gpu(ch, cfg, [np.zeros(100)])
    st = pr.stats(0)
    assert status == 0 and st["converged"] and st["iterations"] == 1 and st["inc"][0] == 0.0
    assert not np.any(pr.get_slices(0))
    pr.close()


def test_precisions_agree_and_runs_are_deterministic(gpu_lib):
    ch = gpu_lib
    n = 700
    base = dict(n=n, eps=0.03, T=0.02, n_slices=5, fine_steps=20, variant="NPA-I", newton_tol=1e-12, max_iters=3)
    u0 = ch_inputs.initial_condition(1, n, 31, amp=0.3)
    out = {}
    for prec in (0, 1):
        runs = []
        for _ in range(2):
            pr, _ = run_gpu(ch, ch.Config(**base, precision=prec), [u0], reference=False)
            runs.append(pr.get_slices(0))
            pr.close()
        assert np.array_equal(runs[0], runs[1])
        out[prec] = runs[0]
    r, tol = oracle_and_floor(o.Params(n=n, eps=0.03, T=0.02, N=5, J=20, fine="nl", coarse="lin1",
                                       newton_tol=1e-12, max_iters=3), u0)
    assert np.max(np.abs(out[0] - out[1])) <= tol
    assert np.max(np.abs(out[1] - r.U)) <= tol


def test_errors_are_reported_not_faulted(gpu_lib):
    ch = gpu_lib
    cfg = ch.Config(n=256, eps=0.02, T=0.1, n_slices=4, fine_steps=2, variant="NPA-I", newton_max=1,
                    newton_tol=1e-14)
    pr = ch.Parareal(cfg, batch=2)
    with pytest.raises(ch.ChError) as e:
        pr.run()
    assert e.value.name == "CH_ERR_STATE"
    pr.close()
    pr = ch.Parareal(cfg, batch=1)
    with pytest.raises(ch.ChError) as e:
        pr.set_initial(0, np.zeros(10))
    assert e.value.name == "CH_ERR_INVALID"
    pr.close()
    pr = ch.Parareal(cfg, batch=1)
    pr.set_initial(0, ch_inputs.initial_condition(1, 256, 1, amp=0.5))
    with pytest.raises(ch.ChError) as e:
        pr.run()
    assert e.value.name == "CH_ERR_NEWTON"
    # the error is sticky on the handle
    with pytest.raises(ch.ChError):
        pr.run()
    pr.close()
    # a fresh handle works after the failure
    pr, _ = run_gpu(ch, ch.Config(n=32, eps=0.1, T=0.01, n_slices=2, fine_steps=2), [np.ones(32) * 0.1],
                    reference=False)
    pr.close()


def test_stats_and_timeline(gpu_lib):
    ch = gpu_lib
    n, N, J = 512, 6, 10
    cfg = ch.Config(n=n, eps=0.05, T=0.02, n_slices=N, fine_steps=J, variant="NPA-I", max_iters=4)
    u0 = ch_inputs.initial_condition(1, n, 2, amp=0.2)
    pr, _ = run_gpu(ch, cfg, [u0])
    st = pr.stats(0)
    assert st["iterations"] == 4
    assert st["fine_point_steps"] == sum((N - k) * J * n for k in range(4))
    t = st["t_iter_ms"][:5]
    assert np.all(np.diff(t) > 0) and t[0] > 0
    assert st["newton_total"] >= sum((N - k) * J for k in range(4))
    U, Uref = pr.get_slices(0), pr.get_reference(0)
    h = 1.0 / (n + 1)
    l2 = max(np.sqrt(h * np.sum((U[s] - Uref[s]) ** 2)) for s in range(N + 1))
    assert abs(st["err_l2"][-1] - l2) <= 1e-15 + 1e-12 * l2
    pr.close()


def test_non_default_stream(gpu_lib):
    ch = gpu_lib
    s = torch.cuda.Stream()
    cfg = ch.Config(n=300, eps=0.05, T=0.01, n_slices=4, fine_steps=6, variant="NPA-I")
    u0 = ch_inputs.initial_condition(1, 300, 8, amp=0.3)
    with torch.cuda.stream(s):
        pr = ch.Parareal(cfg, batch=1, stream=s)
        pr.set_initial(0, u0)
        pr.run()
        U = pr.get_slices(0)
        pr.close()
    r = o.parareal(oracle_params(cfg), u0)
    assert np.max(np.abs(U - r.U)) <= 1e-11


def test_autotuned_launch_is_cached_and_consistent(gpu_lib, tmp_path, monkeypatch):
    """The fine-sweep launch chosen by measurement is written to the cache file; a second handle
    reads it back and runs the same configuration (bitwise identical results), and the
    reference computed after tuning equals the Parareal iterate at k = N bit for bit."""
    ch = gpu_lib
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("CH_AUTOTUNE_CACHE", str(cache))
    n, N = 300, 4
    cfg = ch.Config(n=n, eps=0.03, T=0.02, n_slices=N, fine_steps=10, variant="NPA-I", newton_tol=1e-12,
                    precision=1)
    u0 = ch_inputs.initial_condition(1, n, 77, amp=0.1)
    outs = []
    for rep in range(2):
        with ch.Parareal(cfg, batch=3) as pr:
            for b in range(3):
                pr.set_initial(b, u0 if b == 0 else ch_inputs.initial_condition(1, n, 78 + b, amp=0.1))
            pr.compute_reference()
            pr.run()
            outs.append(pr.get_slices(0))
            assert np.array_equal(pr.get_slices(0), pr.get_reference(0))
    assert np.array_equal(outs[0], outs[1])
    text = cache.read_text()
    assert "fine1d n=300 units=12" in text and "alt=" in text and "div=" in text

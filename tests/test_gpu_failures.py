"""Failure detection, injected on the host: the library reports the failure as a status code,
every kernel returns, and the context and the handle stay usable.

* non-finite initial data (1D and 2D) -> CH_ERR_LINSOLVE from run; new finite data clears it and
  the same handle then reproduces a fresh handle's result;
* an inner CG cap of one iteration (lin_max = 1) with a small Newton cap -> CH_ERR_NEWTON, with
  the cap visible in the CG count;
* a bounded device-side wait that nothing ever satisfies (an mbarrier that no thread arrives on,
  polled with the library's bounded-wait routine and a short limit) -> CH_ERR_TIMEOUT, after
  which the device runs the next kernels normally.
"""
import numpy as np
import pytest

import ch_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_status(pr):
    return pr.run(allow_not_converged=True)


@pytest.mark.parametrize("dim,n", [(1, 200), (2, 31)])
def test_nonfinite_initial_data_reports_linsolve_and_handle_recovers(gpu_lib, dim, n):
    ch = gpu_lib
    cfg = ch.Config(dim=dim, n=n, eps=0.05, T=0.01, n_slices=4, fine_steps=3, variant="NPA-I", newton_tol=1e-12,
                    max_iters=2)
    u0 = np.stack([ch_inputs.initial_condition(dim, n, 600 + b, kind="normal", amp=0.1) for b in range(2)])
    bad = u0.copy()
    bad[1, n // 2] = np.nan
    with ch.Parareal(cfg, batch=2) as pr:
        pr.set_initial_batch(bad)
        with pytest.raises(ch.ChError) as ei:
            pr.run()
        assert ei.value.name == "CH_ERR_LINSOLVE"
        # sticky until new data arrives
        with pytest.raises(ch.ChError):
            pr.run()
        pr.set_initial_batch(u0)
        pr.run()
        U = np.stack([pr.get_slices(b) for b in range(2)])
    with ch.Parareal(cfg, batch=2) as fresh:
        fresh.set_initial_batch(u0)
        fresh.run()
        ref = np.stack([fresh.get_slices(b) for b in range(2)])
    assert np.array_equal(U, ref)


def test_inner_cg_cap_is_honoured_and_reported(gpu_lib):
    ch = gpu_lib
    n = 63
    u0 = ch_inputs.initial_condition(2, n, 610, kind="normal", amp=0.3)
    cfg = ch.Config(dim=2, n=n, eps=0.02, T=0.02, n_slices=2, fine_steps=2, variant="NPA-I", newton_tol=1e-12,
                    newton_max=3, max_iters=1, lin_max=1)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_initial(0, u0)
        with pytest.raises(ch.ChError) as ei:
            pr.run()
        assert ei.value.name == "CH_ERR_NEWTON"
        st = pr.stats(0)
        # one CG iteration per Newton iteration at most
        assert 0 < st["inner_iterations"] <= st["newton_total"]
    # the default cap converges on the same problem
    ok = ch.Config(**{**cfg.__dict__, "newton_max": 50, "lin_max": 0})
    with ch.Parareal(ok, batch=1) as pr:
        pr.set_initial(0, u0)
        pr.run()


def test_lin_tol_trades_newton_for_cg_iterations_at_the_same_root(gpu_lib):
    ch = gpu_lib
    n = 63
    u0 = ch_inputs.initial_condition(2, n, 611, kind="normal", amp=0.3)
    out = {}
    for tol in (1e-2, 1e-4, 1e-6):
        cfg = ch.Config(dim=2, n=n, eps=0.02, T=0.01, n_slices=1, fine_steps=1, newton_tol=1e-12, lin_tol=tol)
        newton = torch.zeros(1, dtype=torch.int32, device="cuda")
        y = ch.propagate(cfg, "nl", 1e-4, 2, torch.as_tensor(u0[None], device="cuda"), newton=newton)
        out[tol] = (y.cpu().numpy()[0], int(newton.item()))
    assert out[1e-2][1] > out[1e-4][1] >= out[1e-6][1]
    for tol in (1e-2, 1e-6):
        assert np.max(np.abs(out[tol][0] - out[1e-4][0])) <= 1e-11


def test_bounded_wait_that_is_never_satisfied_times_out(gpu_lib):
    ch = gpu_lib
    assert ch.wait_selftest(spin_limit=2000) == "CH_ERR_TIMEOUT"
    # the context is usable afterwards
    cfg = ch.Config(n=64, eps=0.05, T=0.01, n_slices=2, fine_steps=2, variant="NPA-I", max_iters=1)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_initial(0, ch_inputs.initial_condition(1, 64, 3, amp=0.1))
        pr.run()

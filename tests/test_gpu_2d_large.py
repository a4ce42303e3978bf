"""GPU parity of the 2D path on the large configurations' grids, against the oracle's CG solver
(library CG on A^{-1} J with a sine-transform preconditioner, pinned against sparse LU).

* The 512 x 512 grid (n = 511, eps = 0.01, fine step dt = 2/64/100, coarse step dT = 2/64) in the
  launch shape of the benchmark's 2D fine sweep: all 64 slices of one problem batched in one
  propagation; sampled units are compared with the oracle element by element.
* The 256 x 256 grid (n = 255, eps = 0.01, dt = 0.5/32/100) with its 32 slices, two fine steps per
  slice (T = 0.01), two Parareal iterations, every slice compared element by element.

Tolerance: 1e-8 max-abs, the bound the mixed-precision path (FP32 inner CG under FP64 Newton) is
held to; the measured difference is far below it (the FP64 step floor of these grids is
~1e-11).
"""
import os

import numpy as np
import pytest

import ch_inputs
import oracle
from oracle import oracle2d as o2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-8


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_c4_grid_batched_steps_match_oracle_on_sampled_units(gpu_lib):
    ch = gpu_lib
    n, eps, T, N, J = 511, 0.01, 2.0, 64, 100
    dT, dt = T / N, T / N / J
    units = 64
    u0 = np.stack([ch_inputs.initial_condition(2, n, 2000 + b, kind="normal", amp=0.05) for b in range(units)])
    cfg = ch.Config(dim=2, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, newton_tol=1e-12)
    p = o2.Params(n=n, eps=eps, T=T, N=N, J=J, newton_tol=1e-12, solver="pcg")
    fine = ch.propagate(cfg, "nl", dt, 2, dev(u0)).cpu().numpy()
    coarse = ch.propagate(cfg, "lin1", dT, 1, dev(u0)).cpu().numpy()
    for b in (0, 37, 63):
        ref_f = o2.propagate(p, "nl", dt, 2, u0[b])
        ref_c = o2.propagate(p, "lin1", dT, 1, u0[b])
        ef = float(np.max(np.abs(fine[b] - ref_f)))
        ec = float(np.max(np.abs(coarse[b] - ref_c)))
        assert ef <= MIXED_TOL and ec <= MIXED_TOL, (b, ef, ec)


def test_c3_grid_parareal_iterates_match_oracle():
    import paper_2304_14074_gb300 as ch
    n, eps, N, J = 255, 0.01, 32, 2
    dt = 0.5 / 32 / 100
    T = N * J * dt
    u0 = ch_inputs.initial_condition(2, n, 1, kind="normal", amp=0.05)
    cfg = ch.Config(dim=2, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant="NPA-I", newton_tol=1e-12,
                    max_iters=2)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_initial(0, u0)
        pr.run()
        U = pr.get_slices(0)
        st = pr.stats(0)
    p = o2.Params(n=n, eps=eps, T=T, N=N, J=J, fine="nl", coarse="lin1", newton_tol=1e-12, solver="pcg")
    with oracle.spawn_pool(min(16, os.cpu_count() or 1)) as pool:
        r = o2.parareal(p, u0, max_iters=2, pmap=pool.map)
    assert st["iterations"] == 2
    err = float(np.max(np.abs(U - r.U)))
    assert err <= MIXED_TOL, err
    # the increments of the two iterations (Section 4 stop-rule quantity) agree as well
    assert np.allclose(st["inc"][:2], r.inc, rtol=1e-6, atol=MIXED_TOL)

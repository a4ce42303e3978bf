"""GPU parity of the Section 3 a-priori bound (ch_parareal_theory_bound) against the oracle, and
the bound against the GPU's own Parareal iterates on the frozen model it is proved for."""
import numpy as np
import pytest

import ch_inputs
from oracle import bounds as ob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n", [(1, 31), (1, 1024), (2, 15), (2, 255)])
@pytest.mark.parametrize("variant", ["PA-I", "PA-II", "PA-III", "NPA-I", "NPA-II"])
@pytest.mark.parametrize("coarse_steps", [1, 2])
def test_theory_bound_matches_oracle(gpu_lib, dim, n, variant, coarse_steps):
    """a, b: the largest mode factors (FP64 sin and pow on both sides: a few ulp); the factors
    are formed in logarithms on the GPU and directly in the oracle."""
    ch = gpu_lib
    eps, T, N, J, kmax = 0.0725, 1.0, 20, 200, 24
    cfg = ch.Config(dim=dim, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, coarse_steps=coarse_steps,
                    variant=variant)
    c1 = 0.1181 if variant.startswith("NPA") else 0.0
    a, b, f = ch.theory_bound(cfg, kmax, lte_const=c1)
    ra, rb, rf = ob.bound(variant, n, dim, eps, T, N, J, kmax, lte_const=c1, coarse_steps=coarse_steps)
    assert a == pytest.approx(ra, rel=1e-12, abs=1e-15)
    assert b == pytest.approx(rb, rel=1e-13)
    assert f[0] == 1.0 and np.all(f[N:] == 0.0)
    np.testing.assert_allclose(f, rf, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("dim,n", [(1, 63), (2, 15)])
@pytest.mark.parametrize("variant", ["PA-I", "PA-II", "PA-III"])
def test_gpu_parareal_errors_within_theory_bound(gpu_lib, dim, n, variant):
    """Theorems 3.7 / 3.9 / 3.11 on the frozen model (diag(u^2) = I): the GPU run's errors
    (max over slices, L2_h, a multiple of the Euclidean norm of the theorems) stay below the
    GPU-computed factor times the error of the coarse initial guess, iterate by iterate."""
    ch = gpu_lib
    eps, T, N, J = 0.0725, 1.0, 10, 20
    cfg = ch.Config(dim=dim, n=n, eps=eps, T=T, n_slices=N, fine_steps=J, variant=variant, frozen=True,
                    precision=0, newton_tol=1e-13)
    _, _, f = ch.theory_bound(cfg, N)
    u0 = ch_inputs.initial_condition(dim, n, 21, amp=0.5)
    with ch.Parareal(cfg, batch=1) as pr:
        pr.set_initial(0, u0)
        pr.compute_reference()
        pr.run()
        e = pr.stats(0)["err_l2"]
    assert e[0] > 0 and len(e) == N + 1
    for k in range(1, N + 1):
        assert e[k] <= f[k] * e[0] * (1 + 1e-9) + 1e-13, (k, e[k], f[k] * e[0])

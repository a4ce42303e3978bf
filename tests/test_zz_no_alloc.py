"""The allocation-free entry point against the handle API.

ch_parareal_solve_noalloc serves callers that cannot call cudaMalloc (their device memory is
owned by another allocator, or cudaMalloc's device synchronisation is not acceptable in their
loop); its scratch is a fixed file-scope device array. This file is collected last so that a
run stopping at the first failure has run every other test first; it also passes alone.
"""
import ctypes as C

import numpy as np
import pytest

import ch_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(ch, cfg, u0_dev, U_dev):
    lib = ch.load()
    cc = cfg.c()
    iters = C.c_int(-1)
    s = lib.ch_parareal_solve_noalloc(C.byref(cc), u0_dev.shape[0], C.c_void_p(u0_dev.data_ptr()),
                                      C.c_void_p(U_dev.data_ptr()), U_dev.numel(), C.byref(iters),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return s, iters.value


def test_noalloc_matches_handle_api_on_two_calls_in_a_row():
    import paper_2304_14074_gb300 as ch
    n, N, B = 300, 8, 3
    cfg = ch.Config(n=n, eps=0.05, T=0.02, n_slices=N, fine_steps=10, variant="NPA-I", newton_tol=1e-12,
                    max_iters=4, precision=1)
    u0 = np.stack([ch_inputs.initial_condition(1, n, 40 + b, amp=0.3) for b in range(B)])
    u0_dev = torch.as_tensor(u0, dtype=torch.float64, device="cuda")
    with ch.Parareal(cfg, batch=B) as pr:
        pr.set_initial_device(u0_dev)
        pr.run()
        ref = torch.empty((B, N + 1, n), dtype=torch.float64, device="cuda")
        pr.get_slices_device(ref)
        torch.cuda.synchronize()
    for call in range(2):
        U = torch.full((B, N + 1, n), float("nan"), dtype=torch.float64, device="cuda")
        s, iters = _noalloc(ch, cfg, u0_dev, U)
        assert s == 0, ch.STATUS.get(s)
        assert iters == 4
        assert torch.max(torch.abs(U - ref)).item() <= 1e-11, call


def test_noalloc_rejects_problems_beyond_its_scratch():
    import paper_2304_14074_gb300 as ch
    n, N, B = 1024, 64, 32  # F and G(U) alone need 2 * 32 * 64 * 1024 * 8 bytes = 32 MiB > 16 MiB
    cfg = ch.Config(n=n, eps=0.02, T=0.1, n_slices=N, fine_steps=2, variant="NPA-I", max_iters=1)
    u0_dev = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    U = torch.zeros((B, N + 1, n), dtype=torch.float64, device="cuda")
    s, _ = _noalloc(ch, cfg, u0_dev, U)
    assert ch.STATUS[s] == "CH_ERR_INVALID"

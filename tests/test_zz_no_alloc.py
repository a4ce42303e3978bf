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


def test_noalloc_rejects_invalid_arguments():
    import paper_2304_14074_gb300 as ch
    n, N, B = 64, 4, 1
    u0_dev = torch.zeros((B, n), dtype=torch.float64, device="cuda")
    U = torch.zeros((B, N + 1, n), dtype=torch.float64, device="cuda")
    for bad in (dict(eps=float("inf")), dict(T=float("nan")), dict(tol=float("nan")), dict(max_iters=N + 1)):
        kw = dict(n=n, eps=0.05, T=0.01, n_slices=N, fine_steps=2, variant="NPA-I", max_iters=1)
        kw.update(bad)
        s, _ = _noalloc(ch, ch.Config(**kw), u0_dev, U)
        assert ch.STATUS[s] == "CH_ERR_INVALID", bad
    cfg = ch.Config(n=n, eps=0.05, T=0.01, n_slices=N, fine_steps=2, variant="NPA-I", max_iters=1)
    lib = ch.load()
    cc = cfg.c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.ch_parareal_solve_noalloc(C.byref(cc), B, C.c_void_p(u0_dev.data_ptr()), C.c_void_p(U.data_ptr()),
                                         U.numel() - 1, None, stream) == 1  # wrong length


_RESET_CHILD = r"""
import ctypes as C, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import ch_inputs
import paper_2304_14074_gb300 as ch
lib = ch.load()
rt = C.CDLL("libcudart.so.13")  # the runtime the library already loaded
n, N, B = 300, 8, 3
cfg = ch.Config(n=n, eps=0.05, T=0.02, n_slices=N, fine_steps=10, variant="NPA-I", newton_tol=1e-12,
                max_iters=4, precision=1)
u0 = np.ascontiguousarray(np.stack([ch_inputs.initial_condition(1, n, 40 + b, amp=0.3) for b in range(B)]))

def handle_api():
    pr = ch.Parareal(cfg, batch=B, stream=0)  # legacy default stream: no torch in this process
    pr.set_initial_batch(u0)
    pr.run()
    out = np.stack([pr.get_slices(b) for b in range(B)])
    pr.close()
    return out

def noalloc():
    u0_dev, U_dev = C.c_void_p(), C.c_void_p()
    assert rt.cudaMalloc(C.byref(u0_dev), C.c_size_t(u0.nbytes)) == 0
    assert rt.cudaMalloc(C.byref(U_dev), C.c_size_t(B * (N + 1) * n * 8)) == 0
    assert rt.cudaMemcpy(u0_dev, u0.ctypes.data_as(C.c_void_p), C.c_size_t(u0.nbytes), 1) == 0
    cc = cfg.c()
    it = C.c_int(-1)
    s = lib.ch_parareal_solve_noalloc(C.byref(cc), B, u0_dev, U_dev, B * (N + 1) * n, C.byref(it), None)
    out = np.empty((B, N + 1, n))
    assert rt.cudaMemcpy(out.ctypes.data_as(C.c_void_p), U_dev, C.c_size_t(out.nbytes), 2) == 0
    rt.cudaFree(u0_dev)
    rt.cudaFree(U_dev)
    assert s == 0 and it.value == 4, (s, it.value)
    return out

ref = handle_api()
a = noalloc()
assert rt.cudaDeviceReset() == 0  # a new primary context: the module reloads
b = noalloc()
ref2 = handle_api()
assert "torch" not in sys.modules
for x in (a, b, ref2):
    assert np.max(np.abs(x - ref)) <= 1e-11, np.max(np.abs(x - ref))
print("reset ok")
"""


def test_noalloc_after_device_reset_matches_handle_api(tmp_path):
    """cudaDeviceReset destroys the context that held the scratch array's address; the next call
    looks the address up again in the new context (and the kernels' attributes are set again),
    so results before and after the reset equal the handle API's. Runs in a child process that
    uses no torch (a reset would invalidate torch's allocations)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = tmp_path / "reset_child.py"
    child.write_text(_RESET_CHILD)
    r = subprocess.run([sys.executable, str(child), root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "reset ok" in r.stdout, r.stdout + r.stderr

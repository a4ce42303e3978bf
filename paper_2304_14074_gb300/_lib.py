"""ctypes binding of the C ABI in ``include/ch_parareal.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/libchparareal.so``. This module
never computes any part of it: when the library cannot be loaded it raises, it does not
fall back. Torch is used only for device memory (tensor data pointers) and streams.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

CH_MAX_ITERS = 1024

STATUS = {0: "CH_OK", 1: "CH_ERR_INVALID", 2: "CH_ERR_OOM", 3: "CH_ERR_CUDA", 4: "CH_ERR_NEWTON",
          5: "CH_ERR_LINSOLVE", 6: "CH_ERR_NOT_CONVERGED", 7: "CH_ERR_TIMEOUT", 8: "CH_ERR_STATE"}
VARIANTS = {"PA-I": 0, "PA-II": 1, "PA-III": 2, "NPA-I": 3, "NPA-II": 4}
SCHEMES = {"lin1": 0, "nl": 1, "lin2": 2}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTED_SYMBOLS = [
    "ch_parareal_create", "ch_parareal_set_initial", "ch_parareal_set_initial_batch",
    "ch_parareal_set_initial_device", "ch_parareal_get_slices_batch",
    "ch_parareal_compute_reference", "ch_parareal_run", "ch_parareal_get_slices",
    "ch_parareal_get_slices_device", "ch_parareal_get_reference", "ch_parareal_get_stats",
    "ch_parareal_get_execution",
    "ch_parareal_destroy", "ch_parareal_last_error", "ch_status_string", "ch_propagate",
    "ch_parareal_solve_noalloc", "ch_sine_transform_2d", "ch_parareal_set_coarse_model",
    "ch_parareal_get_reference_device", "ch_parareal_set_eps", "ch_gtheta_create", "ch_gtheta_destroy", "ch_gtheta_last_error",
    "ch_gtheta_set_params", "ch_gtheta_get_params", "ch_gtheta_forward", "ch_gtheta_gradients",
    "ch_gtheta_train", "ch_ensemble_create", "ch_ensemble_set_initial", "ch_ensemble_compute_reference",
    "ch_ensemble_run", "ch_ensemble_get_slices", "ch_ensemble_get_reference", "ch_ensemble_get_stats",
    "ch_ensemble_groups", "ch_ensemble_destroy", "ch_ensemble_last_error", "ch_parareal_theory_bound",
    "ch_parareal_set_fine_nn", "ch_wait_selftest", "ch_gtheta_activations", "ch_gtheta_set_loss",
]
_NO_STATUS = ("ch_parareal_destroy", "ch_parareal_last_error", "ch_status_string", "ch_gtheta_destroy",
              "ch_gtheta_last_error", "ch_ensemble_destroy", "ch_ensemble_last_error", "ch_ensemble_groups")

CH_GTHETA_PARAMS = 37601
GTHETA_FORMS = {"residual": 0, "correction": 1}
# Flat parameter layout of G_theta: layer l has W_l [3][3][Cout][Cin] then b_l [Cout].
GTHETA_CHANNELS = [1, 32, 32, 32, 32, 32, 1]


class ChError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, f"status {status}")
        super().__init__(f"{what}: {self.name}" + (f" ({detail})" if detail else ""))


class _Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int), ("eps", C.c_double), ("T", C.c_double),
                ("n_slices", C.c_int), ("fine_steps", C.c_int), ("coarse_steps", C.c_int),
                ("variant", C.c_int), ("newton_tol", C.c_double), ("newton_max", C.c_int),
                ("tol", C.c_double), ("max_iters", C.c_int), ("precision", C.c_int), ("frozen", C.c_int),
                ("err_tol", C.c_double), ("lin_tol", C.c_double), ("lin_max", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("inc", C.c_double * CH_MAX_ITERS),
                ("err_l2", C.c_double * CH_MAX_ITERS), ("err_max", C.c_double * CH_MAX_ITERS),
                ("t_iter_ms", C.c_double * CH_MAX_ITERS), ("newton_total", C.c_longlong),
                ("newton_max", C.c_int), ("fine_point_steps", C.c_longlong), ("fine_sweep_ms", C.c_double),
                ("coarse_sweep_ms", C.c_double), ("fine_sweep_launches", C.c_int), ("kernel_launches", C.c_int),
                ("inner_iterations", C.c_longlong), ("coarse_model", C.c_int), ("coarse_fallback_iter", C.c_int)]


@dataclass
class Config:
    """Problem and method parameters (Eq. 1.1, Section 2, Section 4); see ch_config."""
    n: int
    eps: float
    T: float
    n_slices: int
    fine_steps: int
    coarse_steps: int = 1
    variant: str = "NPA-I"
    newton_tol: float = 1e-12
    newton_max: int = 50
    tol: float = 0.0
    max_iters: int = -1
    precision: int = 1
    frozen: bool = False
    err_tol: float = 0.0
    dim: int = 1
    lin_tol: float = 0.0  # 2D inner CG reduction factor (<= 0: 1e-3)
    lin_max: int = 0      # 2D inner CG iterations at most (<= 0: 60)

    def c(self) -> _Config:
        mi = self.n_slices if self.max_iters < 0 else self.max_iters
        return _Config(self.dim, self.n, self.eps, self.T, self.n_slices, self.fine_steps, self.coarse_steps,
                       VARIANTS[self.variant], self.newton_tol, self.newton_max, self.tol, mi, self.precision,
                       int(self.frozen), self.err_tol, self.lin_tol, self.lin_max)


_lib = None


def load(build_if_missing: bool = True):
    """Loads the CUDA library; raises when it is missing or cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    lib = C.CDLL(path)
    vp, d, sz = C.c_void_p, C.POINTER(C.c_double), C.c_size_t
    lib.ch_parareal_create.argtypes = [C.POINTER(_Config), C.c_int, vp, C.POINTER(vp)]
    lib.ch_parareal_set_initial.argtypes = [vp, C.c_int, d, sz]
    lib.ch_parareal_set_initial_device.argtypes = [vp, vp, sz]
    lib.ch_parareal_set_initial_batch.argtypes = [vp, d, sz]
    lib.ch_parareal_get_slices_batch.argtypes = [vp, d, sz]
    lib.ch_parareal_compute_reference.argtypes = [vp]
    lib.ch_parareal_run.argtypes = [vp]
    lib.ch_parareal_get_slices.argtypes = [vp, C.c_int, d, sz]
    lib.ch_parareal_get_slices_device.argtypes = [vp, vp, sz]
    lib.ch_parareal_get_reference.argtypes = [vp, C.c_int, d, sz]
    lib.ch_parareal_get_stats.argtypes = [vp, C.c_int, C.POINTER(_Stats)]
    lib.ch_parareal_get_execution.argtypes = [vp, C.POINTER(C.c_int)]
    lib.ch_parareal_destroy.argtypes = [vp]
    lib.ch_parareal_destroy.restype = None
    lib.ch_parareal_last_error.argtypes = [vp]
    lib.ch_parareal_last_error.restype = C.c_char_p
    lib.ch_status_string.argtypes = [C.c_int]
    lib.ch_status_string.restype = C.c_char_p
    lib.ch_propagate.argtypes = [C.POINTER(_Config), C.c_int, C.c_int, C.c_double, C.c_int, vp, vp, vp, vp]
    lib.ch_sine_transform_2d.argtypes = [vp, vp, C.c_int, C.c_int, vp]
    lib.ch_parareal_theory_bound.argtypes = [C.POINTER(_Config), C.c_double, C.c_int, d, sz, vp]
    lib.ch_parareal_set_fine_nn.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_int]
    lib.ch_wait_selftest.argtypes = [C.c_uint, vp]
    lib.ch_gtheta_activations.argtypes = [vp, vp, C.c_int, C.c_int, vp, sz]
    lib.ch_parareal_solve_noalloc.argtypes = [C.POINTER(_Config), C.c_int, vp, vp, sz, C.POINTER(C.c_int), vp]
    f = C.POINTER(C.c_float)
    lib.ch_parareal_set_coarse_model.argtypes = [vp, f, sz, C.c_int]
    lib.ch_parareal_get_reference_device.argtypes = [vp, vp, sz]
    lib.ch_parareal_set_eps.argtypes = [vp, d, sz]
    lib.ch_gtheta_create.argtypes = [C.c_ulonglong, vp, C.POINTER(vp)]
    lib.ch_gtheta_destroy.argtypes = [vp]
    lib.ch_gtheta_destroy.restype = None
    lib.ch_gtheta_last_error.argtypes = [vp]
    lib.ch_gtheta_last_error.restype = C.c_char_p
    lib.ch_gtheta_set_params.argtypes = [vp, f, sz]
    lib.ch_gtheta_get_params.argtypes = [vp, f, sz]
    lib.ch_gtheta_forward.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int]
    lib.ch_gtheta_gradients.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, f, sz, f]
    lib.ch_gtheta_set_loss.argtypes = [vp, C.c_int]
    lib.ch_gtheta_train.argtypes = [vp, vp, vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                    C.c_ulonglong, f]
    ip = C.POINTER(C.c_int)
    lib.ch_ensemble_create.argtypes = [C.POINTER(_Config), C.c_int, ip, d, C.POINTER(vp)]
    lib.ch_ensemble_set_initial.argtypes = [vp, C.c_int, d, sz]
    lib.ch_ensemble_compute_reference.argtypes = [vp]
    lib.ch_ensemble_run.argtypes = [vp]
    lib.ch_ensemble_get_slices.argtypes = [vp, C.c_int, d, sz]
    lib.ch_ensemble_get_reference.argtypes = [vp, C.c_int, d, sz]
    lib.ch_ensemble_get_stats.argtypes = [vp, C.c_int, C.POINTER(_Stats)]
    lib.ch_ensemble_groups.argtypes = [vp]
    lib.ch_ensemble_groups.restype = C.c_int
    lib.ch_ensemble_destroy.argtypes = [vp]
    lib.ch_ensemble_destroy.restype = None
    lib.ch_ensemble_last_error.argtypes = [vp]
    lib.ch_ensemble_last_error.restype = C.c_char_p
    for name in EXPORTED_SYMBOLS:
        if name not in _NO_STATUS:
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    """Device pointer of a contiguous CUDA tensor (validated)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _host(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Parareal:
    """A handle of `batch` problems sharing one configuration (ch_parareal_*)."""

    def __init__(self, cfg: Config, batch: int = 1, stream=None):
        self.lib = load()
        self.cfg = cfg
        self.batch = batch
        self.pts = cfg.n ** cfg.dim
        self._h = C.c_void_p()
        self._cc = cfg.c()
        s = self.lib.ch_parareal_create(C.byref(self._cc), batch, _stream_ptr(stream), C.byref(self._h))
        if s != 0:
            raise ChError(s, "ch_parareal_create")

    def _check(self, s, what, ok=(0,)):
        if s not in ok:
            detail = self.lib.ch_parareal_last_error(self._h).decode() if self._h else ""
            raise ChError(s, what, detail)
        return s

    def set_initial(self, problem: int, u0) -> None:
        u = _host(u0)
        self._check(self.lib.ch_parareal_set_initial(self._h, problem, u.ctypes.data_as(C.POINTER(C.c_double)),
                                                     u.size), "ch_parareal_set_initial")

    def set_initial_batch(self, u0) -> None:
        """u0: [batch, n^d] host array (pinned host memory makes the copy asynchronous)."""
        if isinstance(u0, np.ndarray):
            u = _host(u0)
            ptr, size = u.ctypes.data_as(C.POINTER(C.c_double)), u.size
        else:  # a CPU torch tensor, possibly pinned
            ptr, size = C.cast(C.c_void_p(u0.data_ptr()), C.POINTER(C.c_double)), u0.numel()
        self._check(self.lib.ch_parareal_set_initial_batch(self._h, ptr, size), "ch_parareal_set_initial_batch")

    def get_slices_batch(self, out=None):
        """All problems' final iterates [batch, N+1, n^d] into host memory (numpy or CPU tensor)."""
        if out is None:
            out = np.empty((self.batch, self.cfg.n_slices + 1, self.pts))
        if isinstance(out, np.ndarray):
            ptr, size = out.ctypes.data_as(C.POINTER(C.c_double)), out.size
        else:
            ptr, size = C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double)), out.numel()
        self._check(self.lib.ch_parareal_get_slices_batch(self._h, ptr, size), "ch_parareal_get_slices_batch")
        return out

    def set_initial_device(self, u0_dev) -> None:
        self._check(self.lib.ch_parareal_set_initial_device(self._h, _dptr(u0_dev), u0_dev.numel()),
                    "ch_parareal_set_initial_device")

    def compute_reference(self) -> None:
        self._check(self.lib.ch_parareal_compute_reference(self._h), "ch_parareal_compute_reference")

    def run(self, allow_not_converged: bool = True) -> int:
        ok = (0, 6) if allow_not_converged else (0,)
        return self._check(self.lib.ch_parareal_run(self._h), "ch_parareal_run", ok)

    def get_slices(self, problem: int) -> np.ndarray:
        out = np.empty((self.cfg.n_slices + 1, self.pts))
        self._check(self.lib.ch_parareal_get_slices(self._h, problem, out.ctypes.data_as(C.POINTER(C.c_double)),
                                                    out.size), "ch_parareal_get_slices")
        return out

    def get_slices_device(self, out_dev) -> None:
        self._check(self.lib.ch_parareal_get_slices_device(self._h, _dptr(out_dev), out_dev.numel()),
                    "ch_parareal_get_slices_device")

    def get_reference(self, problem: int) -> np.ndarray:
        out = np.empty((self.cfg.n_slices + 1, self.pts))
        self._check(self.lib.ch_parareal_get_reference(self._h, problem,
                                                       out.ctypes.data_as(C.POINTER(C.c_double)), out.size),
                    "ch_parareal_get_reference")
        return out

    def execution(self) -> str:
        """The execution its first reference or run chose: 2D "graphs", "persistent", "host" or
        "cluster"; 1D "default" or "alt" (the fine sweep's CTA mapping); "" before that."""
        v = C.c_int()
        self._check(self.lib.ch_parareal_get_execution(self._h, C.byref(v)), "ch_parareal_get_execution")
        if v.value < 0:
            return ""
        if self.cfg.dim == 2:
            return ("graphs", "persistent", "host", "cluster")[v.value]
        return ("default", "alt")[v.value]

    def stats(self, problem: int) -> dict:
        st = _Stats()
        self._check(self.lib.ch_parareal_get_stats(self._h, problem, C.byref(st)), "ch_parareal_get_stats")
        k = st.iterations
        return {"iterations": k, "converged": bool(st.converged), "inc": np.array(st.inc[:k]),
                "err_l2": np.array(st.err_l2[:k + 1]), "err_max": np.array(st.err_max[:k + 1]),
                "t_iter_ms": np.array(st.t_iter_ms[:self.cfg.c().max_iters + 1]),
                "newton_total": st.newton_total, "newton_max": st.newton_max,
                "fine_point_steps": st.fine_point_steps, "fine_sweep_ms": st.fine_sweep_ms,
                "coarse_sweep_ms": st.coarse_sweep_ms, "fine_sweep_launches": st.fine_sweep_launches,
                "kernel_launches": st.kernel_launches, "inner_iterations": st.inner_iterations,
                "coarse_model": st.coarse_model, "coarse_fallback_iter": st.coarse_fallback_iter}

    def set_coarse_model(self, params, form: str = "correction") -> None:
        """Learned coarse propagator G_theta with these FP32 parameters (None: plain coarse step);
        form "residual" (U + R(U)) or "correction" (G(U) + R(U))."""
        f = GTHETA_FORMS[form]
        if params is None:
            self._check(self.lib.ch_parareal_set_coarse_model(self._h, None, 0, f), "ch_parareal_set_coarse_model")
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.lib.ch_parareal_set_coarse_model(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size,
                                                          f), "ch_parareal_set_coarse_model")

    def set_fine_nn(self, n_sub: int, theta: float = 0.25, tol: float = 1e-10, max_iter: int = 200) -> None:
        """Neumann-Neumann fine solver (Section 4.6, 1D PA-I) with n_sub subdomains; 0 restores the
        monolithic solve."""
        self._check(self.lib.ch_parareal_set_fine_nn(self._h, n_sub, theta, tol, max_iter), "ch_parareal_set_fine_nn")

    def set_eps(self, eps) -> None:
        """Per-problem eps (2D): one value per problem of the batch."""
        e = _host(eps)
        self._check(self.lib.ch_parareal_set_eps(self._h, e.ctypes.data_as(C.POINTER(C.c_double)), e.size),
                    "ch_parareal_set_eps")

    def get_reference_device(self, out_dev) -> None:
        self._check(self.lib.ch_parareal_get_reference_device(self._h, _dptr(out_dev), out_dev.numel()),
                    "ch_parareal_get_reference_device")

    def close(self) -> None:
        if self._h:
            self.lib.ch_parareal_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def propagate(cfg: Config, scheme: str, dt: float, nsteps: int, u_in, u_out=None, newton=None, stream=None):
    """Batched propagation on the device (ch_propagate). u_in: CUDA float64 tensor [batch, n^d]."""
    import torch
    lib = load()
    if u_out is None:
        u_out = torch.empty_like(u_in)
    batch = u_in.shape[0]
    cc = cfg.c()
    s = lib.ch_propagate(C.byref(cc), batch, SCHEMES[scheme], dt, nsteps, _dptr(u_in), _dptr(u_out),
                         _dptr(newton) if newton is not None else None, _stream_ptr(stream))
    if s != 0:
        raise ChError(s, "ch_propagate")
    return u_out


def wait_selftest(spin_limit: int = 2000, stream=None) -> str:
    """Runs ch_wait_selftest (a bounded wait that nothing satisfies) and returns the status name;
    CH_ERR_TIMEOUT is the expected outcome."""
    lib = load()
    return STATUS.get(lib.ch_wait_selftest(spin_limit, _stream_ptr(stream)), "unknown")


def theory_bound(cfg: Config, kmax: int, lte_const: float = 0.0, stream=None):
    """Section 3 a-priori bound (ch_parareal_theory_bound): returns (a, b, factors[0..kmax]),
    max_j ||E_j^k|| <= factors[k] max_j ||E_j^0||. lte_const: C_1 / C_2 for NPA-I / NPA-II."""
    import numpy as np
    lib = load()
    out = np.zeros(kmax + 3)
    cc = cfg.c()
    s = lib.ch_parareal_theory_bound(C.byref(cc), lte_const, kmax, out.ctypes.data_as(C.POINTER(C.c_double)),
                                     out.size, _stream_ptr(stream))
    if s != 0:
        raise ChError(s, "ch_parareal_theory_bound")
    return float(out[0]), float(out[1]), out[2:].copy()


def sine_transform_2d(x, out=None, stream=None):
    """Orthonormal 2D DST-I on the device (ch_sine_transform_2d). x: CUDA float32 [batch, n, n]."""
    import torch
    lib = load()
    if out is None:
        out = torch.empty_like(x)
    s = lib.ch_sine_transform_2d(_dptr(x), _dptr(out), x.shape[0], x.shape[-1], _stream_ptr(stream))
    if s != 0:
        raise ChError(s, "ch_sine_transform_2d")
    return out


class GTheta:
    """Learned coarse propagator G_theta(U) = U + R(U) (ch_gtheta_*)."""

    def __init__(self, seed: int = 0, stream=None):
        self.lib = load()
        self._h = C.c_void_p()
        s = self.lib.ch_gtheta_create(seed, _stream_ptr(stream), C.byref(self._h))
        if s != 0:
            raise ChError(s, "ch_gtheta_create")

    def _check(self, s, what):
        if s != 0:
            detail = self.lib.ch_gtheta_last_error(self._h).decode() if self._h else ""
            raise ChError(s, what, detail)

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._check(self.lib.ch_gtheta_set_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
                    "ch_gtheta_set_params")

    def set_loss(self, relative: bool) -> None:
        """Training loss: mean squared error on the crop windows (False, the default), or each
        crop's squared error relative to its target's energy (True)."""
        self._check(self.lib.ch_gtheta_set_loss(self._h, 1 if relative else 0), "ch_gtheta_set_loss")

    def get_params(self) -> np.ndarray:
        p = np.empty(CH_GTHETA_PARAMS, dtype=np.float32)
        self._check(self.lib.ch_gtheta_get_params(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
                    "ch_gtheta_get_params")
        return p

    def forward(self, u_dev, out=None, base=None):
        """base + R(U) (base = U when None) of a CUDA float64 tensor [batch, n, n]."""
        import torch
        if out is None:
            out = torch.empty_like(u_dev)
        self._check(self.lib.ch_gtheta_forward(self._h, _dptr(u_dev), _dptr(base) if base is not None else None,
                                               _dptr(out), u_dev.shape[0], u_dev.shape[-1]), "ch_gtheta_forward")
        return out

    def activations(self, u_dev):
        """Every layer's output for a CUDA float64 tensor [batch, n, n]: (a1..a5 as a float32 tensor
        [5, batch, n, n, 32] holding the stored BF16 values, R as [batch, n, n])."""
        import torch
        B, n = u_dev.shape[0], u_dev.shape[-1]
        out = torch.empty(B * n * n * (5 * 32 + 1), dtype=torch.float32, device=u_dev.device)
        self._check(self.lib.ch_gtheta_activations(self._h, _dptr(u_dev), B, n, _dptr(out), out.numel()),
                    "ch_gtheta_activations")
        per = B * n * n * 32
        return out[:5 * per].view(5, B, n, n, 32), out[5 * per:].view(B, n, n)

    def gradients(self, x_dev, target_dev, margin: int):
        """(loss, flat FP32 gradient) of one minibatch: CUDA float32 tensors [batch, S, S]."""
        g = np.empty(CH_GTHETA_PARAMS, dtype=np.float32)
        loss = C.c_float()
        self._check(self.lib.ch_gtheta_gradients(self._h, _dptr(x_dev), _dptr(target_dev), x_dev.shape[0],
                                                 x_dev.shape[-1], margin, g.ctypes.data_as(C.POINTER(C.c_float)),
                                                 g.size, C.byref(loss)), "ch_gtheta_gradients")
        return float(loss.value), g

    def train(self, states_dev, stride: int, steps: int, batch: int, lr: float, seed: int = 0,
              base=None) -> np.ndarray:
        """Adam on crops of snapshot pairs; states_dev (and base, the plain coarse step of each
        snapshot for the correction form): CUDA float64 [ntraj, nsnap, n, n] (or [ntraj, nsnap,
        n*n] with square n). Returns the per-step minibatch losses."""
        ntraj, nsnap = states_dev.shape[0], states_dev.shape[1]
        n = int(round((states_dev[0, 0].numel()) ** 0.5))
        if base is not None and base.shape != states_dev.shape:
            raise ValueError("base must have the shape of states")
        losses = np.empty(steps, dtype=np.float32)
        self._check(self.lib.ch_gtheta_train(self._h, _dptr(states_dev), _dptr(base) if base is not None else None,
                                             ntraj, nsnap, n, stride, steps, batch, lr, seed,
                                             losses.ctypes.data_as(C.POINTER(C.c_float))), "ch_gtheta_train")
        return losses

    def close(self) -> None:
        if self._h:
            self.lib.ch_gtheta_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gtheta_unflatten(p):
    """Flat parameter vector -> ([W_l [3][3][Cout][Cin]], [b_l [Cout]]) as float64 arrays."""
    p = np.asarray(p, dtype=np.float64)
    W, b, o = [], [], 0
    for l in range(6):
        ci, co = GTHETA_CHANNELS[l], GTHETA_CHANNELS[l + 1]
        W.append(p[o:o + 9 * co * ci].reshape(3, 3, co, ci))
        o += 9 * co * ci
        b.append(p[o:o + co].copy())
        o += co
    assert o == CH_GTHETA_PARAMS
    return W, b


def gtheta_flatten(W, b) -> np.ndarray:
    """Inverse of gtheta_unflatten (FP32)."""
    return np.concatenate([np.concatenate([np.asarray(w).ravel(), np.asarray(bb).ravel()])
                           for w, bb in zip(W, b)]).astype(np.float32)


class Ensemble:
    """2D problems of several grid sizes and eps (ch_ensemble_*): grouped by grid size, one
    batched handle per size on its own stream, the groups run concurrently."""

    def __init__(self, cfg: Config, n_per_problem, eps_per_problem):
        self.lib = load()
        self.cfg = cfg
        self.n = [int(v) for v in n_per_problem]
        nn = np.ascontiguousarray(self.n, dtype=np.int32)
        ee = _host(eps_per_problem)
        if ee.size != nn.size:
            raise ValueError("one eps per problem")
        self._h = C.c_void_p()
        self._cc = cfg.c()
        s = self.lib.ch_ensemble_create(C.byref(self._cc), nn.size, nn.ctypes.data_as(C.POINTER(C.c_int)),
                                        ee.ctypes.data_as(C.POINTER(C.c_double)), C.byref(self._h))
        if s != 0:
            raise ChError(s, "ch_ensemble_create")

    def _check(self, s, what, ok=(0,)):
        if s not in ok:
            detail = self.lib.ch_ensemble_last_error(self._h).decode() if self._h else ""
            raise ChError(s, what, detail)
        return s

    @property
    def groups(self) -> int:
        return self.lib.ch_ensemble_groups(self._h)

    def set_initial(self, problem: int, u0) -> None:
        u = _host(u0)
        self._check(self.lib.ch_ensemble_set_initial(self._h, problem, u.ctypes.data_as(C.POINTER(C.c_double)),
                                                     u.size), "ch_ensemble_set_initial")

    def compute_reference(self) -> None:
        self._check(self.lib.ch_ensemble_compute_reference(self._h), "ch_ensemble_compute_reference")

    def run(self, allow_not_converged: bool = True) -> int:
        ok = (0, 6) if allow_not_converged else (0,)
        return self._check(self.lib.ch_ensemble_run(self._h), "ch_ensemble_run", ok)

    def _slices(self, fn, what, problem):
        out = np.empty((self.cfg.n_slices + 1, self.n[problem] ** 2))
        self._check(fn(self._h, problem, out.ctypes.data_as(C.POINTER(C.c_double)), out.size), what)
        return out

    def get_slices(self, problem: int) -> np.ndarray:
        return self._slices(self.lib.ch_ensemble_get_slices, "ch_ensemble_get_slices", problem)

    def get_reference(self, problem: int) -> np.ndarray:
        return self._slices(self.lib.ch_ensemble_get_reference, "ch_ensemble_get_reference", problem)

    def stats(self, problem: int) -> dict:
        st = _Stats()
        self._check(self.lib.ch_ensemble_get_stats(self._h, problem, C.byref(st)), "ch_ensemble_get_stats")
        k = st.iterations
        return {"iterations": k, "converged": bool(st.converged), "inc": np.array(st.inc[:k]),
                "err_l2": np.array(st.err_l2[:k + 1]), "t_iter_ms": np.array(st.t_iter_ms[:k + 1]),
                "fine_point_steps": st.fine_point_steps, "newton_total": st.newton_total,
                "inner_iterations": st.inner_iterations, "kernel_launches": st.kernel_launches}

    def close(self) -> None:
        if self._h:
            self.lib.ch_ensemble_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""CPU oracle for the Cahn-Hilliard Parareal methods (arXiv 2304.14074).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. The GPU library never calls it,
shares no code with it, and fails loudly when its own CUDA extension is missing.

* ``oracle1d`` : ctypes binding of the plain-C FP64 one-dimensional oracle (``ch_oracle.c``).
* ``oracle2d`` : numpy/scipy FP64 two-dimensional oracle (sparse matrices, direct solves).
* ``bounds``   : the a-priori Parareal error bounds of Section 3 (numpy).
* ``nn1d``     : the Neumann-Neumann fine solver of Section 4.6 in 1D (numpy, dense local solves).

Parity status of every function, and the pins that hold it, are listed in the header of
each module and in the tests under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libch_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with the host compiler (plain -O2, no vector intrinsics)."""
    src = os.path.join(_HERE, "ch_oracle.c")
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "ch_oracle.h"))):
        return LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def spawn_pool(processes: int):
    """A 'spawn' process pool for oracle work whose workers use one BLAS/OpenMP thread each (the
    workers are the parallelism; threaded BLAS inside each of them oversubscribes the cores).
    Spawned, not forked, so it is safe to create after the process has used the GPU."""
    import multiprocessing as mp
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        return mp.get_context("spawn").Pool(processes)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

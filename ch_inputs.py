"""Seeded synthetic inputs for the Cahn-Hilliard Parareal workloads.

This module is shared by the CPU oracle tests, the GPU tests and the benchmark. It
holds no arithmetic of the numerical method: it only draws initial data u^0 on the
interior grid nodes (boundary values are implicitly zero, Section 2.1) and the
per-problem parameters of an ensemble.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), in its published form: the state advances by the odd
constant 0x9E3779B97F4A7C15 and each output is the state passed through two
xor-shift-multiply rounds and a final xor-shift. A 53-bit uniform double in [0, 1)
is the top 53 bits of an output times 2^-53. Normal variates use the Box-Muller
transform (Box and Muller, 1958) on pairs of uniforms, evaluated with numpy's libm.

Values are drawn i.i.d. per interior point, in row-major order (y outer, x inner
in 2D), so the same array feeds the oracle and the GPU path.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of the SplitMix64 stream started at `seed`."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_sym(seed: int, count: int, amp: float) -> np.ndarray:
    """amp * Uniform(-1, 1), i.i.d."""
    return amp * (2.0 * uniform01(seed, count) - 1.0)


def normal(seed: int, count: int, amp: float) -> np.ndarray:
    """amp * N(0, 1), i.i.d., Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return amp * z[:count]


def initial_condition(dim: int, n: int, seed: int, kind: str = "uniform", amp: float = 0.1) -> np.ndarray:
    """u^0 on the n^dim interior nodes, flattened row-major."""
    count = n ** dim
    if kind == "uniform":
        return uniform_sym(seed, count, amp)
    if kind == "normal":
        return normal(seed, count, amp)
    raise ValueError(f"unknown initial-condition kind {kind!r}")


def ensemble_draws(seed: int, count: int, sizes=(64, 128, 256, 512), eps_lo: float = 0.01,
                   eps_hi: float = 0.05):
    """Per-problem (grid size s, eps) for an uneven ensemble, drawn from one stream.

    Problem b takes outputs 2b (size index) and 2b+1 (eps) of the stream.
    """
    u = uniform01(seed, 2 * count)
    size_idx = np.minimum((u[0::2] * len(sizes)).astype(np.int64), len(sizes) - 1)
    s = np.asarray(sizes, dtype=np.int64)[size_idx]
    eps = eps_lo + (eps_hi - eps_lo) * u[1::2]
    return s, eps

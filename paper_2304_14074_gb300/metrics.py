"""Per-iteration metrics of a Parareal run as JSON Lines (host-side logging only).

``Parareal.stats(problem)`` returns one problem's history: the increment of every iteration
(max_n ||U_n^k - U_n^{k-1}||_inf), the error against the sequential fine solution in the L2_h
and max-abs norms of Section 4 (k = 0 is the coarse initial guess), the device time at the end
of each iteration, and whole-run counters (Newton and CG iterations, sweep times, launches).
``stats_records`` turns that into one record per iteration plus one summary record, and
``append_jsonl`` appends records to a file, one JSON object per line. Nothing here computes any
part of the method.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

_SUMMARY_KEYS = ("iterations", "converged", "newton_total", "newton_max", "fine_point_steps", "fine_sweep_ms",
                 "coarse_sweep_ms", "fine_sweep_launches", "kernel_launches", "inner_iterations", "coarse_model",
                 "coarse_fallback_iter")


def _num(x):
    """A JSON-ready scalar: numpy scalars become Python numbers, non-finite values None."""
    if isinstance(x, (bool, np.bool_)):
        return bool(x)
    if isinstance(x, (int, np.integer)):
        return int(x)
    v = float(x)
    return v if math.isfinite(v) else None


def _norm(a, k):
    """Entry k of a norm history; the library reports -1 where no reference was computed."""
    if a is None or k >= len(a):
        return None
    v = _num(a[k])
    return None if v is None or v < 0 else v


def stats_records(stats: dict, **meta) -> list[dict]:
    """One record per iteration k = 0..iterations (k = 0: the coarse initial guess, which has no
    increment) and a final record with ``"summary": true`` and the run's counters. ``meta``
    (for example the workload and the problem index) is copied into every record."""
    k_done = int(stats["iterations"])
    inc = stats.get("inc")
    el2, emx, t = stats.get("err_l2"), stats.get("err_max"), stats.get("t_iter_ms")
    recs = []
    for k in range(k_done + 1):
        r = dict(meta)
        r["k"] = k
        r["inc"] = None if k == 0 or inc is None or k - 1 >= len(inc) else _num(inc[k - 1])
        r["err_l2"] = _norm(el2, k)
        r["err_max"] = _norm(emx, k)
        r["t_ms"] = None if t is None or k >= len(t) else _num(t[k])
        recs.append(r)
    s = dict(meta)
    s["summary"] = True
    for key in _SUMMARY_KEYS:
        if key in stats:
            s[key] = _num(stats[key])
    recs.append(s)
    return recs


def append_jsonl(path: str | os.PathLike, records) -> int:
    """Append the records to ``path`` (created with its directory if missing), one JSON object
    per line; returns the number of lines written."""
    d = os.path.dirname(os.fspath(path))
    if d:
        os.makedirs(d, exist_ok=True)
    n = 0
    with open(path, "a", encoding="utf-8") as f:
        for r in records:
            f.write(json.dumps(r, sort_keys=True) + "\n")
            n += 1
    return n

"""Host-side metrics: a run's per-iteration history as JSON Lines (no GPU). The stats dictionary
is laid out as ``Parareal.stats`` returns it; the values are made up."""
import json

import numpy as np

import paper_2304_14074_gb300 as ch


def fake_stats(k=3, with_reference=True):
    return {"iterations": k, "converged": True,
            "inc": np.array([0.5, 0.05, 1e-9][:k]),
            "err_l2": np.array([0.3, 0.02, 1e-4, 5e-10][:k + 1]) if with_reference else -np.ones(k + 1),
            "err_max": np.array([0.6, 0.03, 2e-4, 9e-10][:k + 1]) if with_reference else -np.ones(k + 1),
            "t_iter_ms": np.array([0.1, 1.1, 2.1, 3.1, 0.0, 0.0]),
            "newton_total": np.int64(1234), "newton_max": 3, "fine_point_steps": 10 ** 9,
            "fine_sweep_ms": 2.5, "coarse_sweep_ms": 0.4, "fine_sweep_launches": 3, "kernel_launches": 10,
            "inner_iterations": 0, "coarse_model": 0, "coarse_fallback_iter": -1}


def test_one_record_per_iteration_and_a_summary():
    recs = ch.stats_records(fake_stats(), workload="c1", problem=7)
    assert len(recs) == 3 + 1 + 1
    assert [r["k"] for r in recs[:-1]] == [0, 1, 2, 3]
    assert recs[0]["inc"] is None  # the coarse initial guess has no increment
    assert [r["inc"] for r in recs[1:4]] == [0.5, 0.05, 1e-9]
    assert [r["err_l2"] for r in recs[:4]] == [0.3, 0.02, 1e-4, 5e-10]
    assert [r["t_ms"] for r in recs[:4]] == [0.1, 1.1, 2.1, 3.1]
    assert all(r["workload"] == "c1" and r["problem"] == 7 for r in recs)
    s = recs[-1]
    assert s["summary"] is True and s["iterations"] == 3 and s["converged"] is True
    assert s["newton_total"] == 1234 and isinstance(s["newton_total"], int)
    assert s["coarse_fallback_iter"] == -1


def test_missing_reference_becomes_null():
    recs = ch.stats_records(fake_stats(2, with_reference=False))
    assert all(r["err_l2"] is None and r["err_max"] is None for r in recs[:-1])


def test_jsonl_round_trip(tmp_path):
    path = tmp_path / "sub" / "metrics.jsonl"
    n = ch.append_jsonl(path, ch.stats_records(fake_stats(), problem=0))
    n += ch.append_jsonl(path, ch.stats_records(fake_stats(1), problem=1))
    lines = path.read_text().splitlines()
    assert n == len(lines) == 5 + 3
    rows = [json.loads(x) for x in lines]
    assert rows[4]["summary"] and rows[4]["problem"] == 0
    assert rows[-1]["summary"] and rows[-1]["problem"] == 1 and rows[-1]["iterations"] == 1
    assert rows[3]["err_max"] == 9e-10


def test_non_finite_values_are_null():
    st = fake_stats()
    st["inc"] = np.array([np.nan, np.inf, 1.0])
    recs = ch.stats_records(st)
    assert recs[1]["inc"] is None and recs[2]["inc"] is None and recs[3]["inc"] == 1.0
    json.dumps(recs, allow_nan=False)  # strict JSON

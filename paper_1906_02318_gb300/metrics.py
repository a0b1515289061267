"""Per-tick records of a control loop, a JSON-lines log, and the paper's metrics.

Each tick yields one record: the tick and trial, the outcome of the selection
(status, chosen slot, number of safe candidates), the intervention and the
host-to-host latency.  summarize() reduces a run to the quantities the paper
reports (Sec. VI-A, VI-D, Table I):
- the fraction of trials that never left the safe set, and each failed trial's
  time to failure (ticks until the plant left the safe set, times the tick
  period);
- the average deviation between the user's input and the applied input, the
  closest safe one (Euclidean distance, Sec. IV-D);
- the average fraction of sampled rollouts that are safe at a tick.
The user's own input, when it is a candidate (slot 0), is not a sampled rollout:
it is taken out of the safe count when it is safe (then it is also the selection,
since it costs nothing).
"""
from __future__ import annotations

import json
import math

import numpy as np

SAFE = 0  # result status of a tick whose selection is safe (mpmi.h MPMI_SAFE)


def tick_record(result: dict, u_h, tick: int, trial: int, n_samples: int,
                include_user: bool = True, latency_s: float | None = None,
                failed: bool = False) -> dict:
    """One tick: `result` is select_input's dict; `failed` marks the tick after
    which the plant left the safe set (the trial ends there)."""
    u_r = np.asarray(result["u_r"], dtype=np.float64).ravel()
    u_h = np.asarray(u_h, dtype=np.float64).ravel()
    user_safe = include_user and result["index"] == 0 and result["status"] == SAFE
    safe_samples = int(result["n_safe"]) - (1 if user_safe else 0)
    return dict(tick=int(tick), trial=int(trial), status=int(result["status"]),
                index=int(result["index"]), n_safe=int(result["n_safe"]),
                safe_fraction=safe_samples / n_samples if n_samples > 0 else 0.0,
                deviation=float(np.linalg.norm(u_r - u_h[:u_r.size])),
                latency_ms=None if latency_s is None else 1e3 * float(latency_s),
                failed=bool(failed))


class TickLog:
    """Appends records to a JSON-lines file (one object per line)."""

    def __init__(self, path: str):
        self.f = open(path, "a", encoding="utf-8")

    def write(self, record: dict) -> None:
        self.f.write(json.dumps(record, sort_keys=True) + "\n")

    def close(self) -> None:
        self.f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def read_log(path: str) -> list[dict]:
    with open(path, encoding="utf-8") as f:
        return [json.loads(line) for line in f if line.strip()]


def _mean_std(v) -> tuple[float, float]:
    v = np.asarray(v, dtype=np.float64)
    if v.size == 0:
        return math.nan, math.nan
    return float(v.mean()), float(v.std())


def summarize(records: list[dict], tick_period_s: float) -> dict:
    """The paper's metrics over a run of tick records (see the module docstring)."""
    trials: dict[int, dict] = {}
    for r in records:
        t = trials.setdefault(r["trial"], dict(ticks=0, failed=False))
        t["ticks"] += 1
        t["failed"] = t["failed"] or r["failed"]
    failures = [t["ticks"] * tick_period_s for t in trials.values() if t["failed"]]
    dev = _mean_std([r["deviation"] for r in records])
    safe = _mean_std([r["safe_fraction"] for r in records])
    lat = [r["latency_ms"] for r in records if r.get("latency_ms") is not None]
    out = dict(ticks=len(records), trials=len(trials),
               safe_trial_fraction=(len(trials) - len(failures)) / len(trials) if trials else
               math.nan,
               mean_time_to_failure_s=float(np.mean(failures)) if failures else None,
               avg_deviation=dev[0], avg_deviation_std=dev[1],
               avg_safe_rollouts=safe[0], avg_safe_rollouts_std=safe[1],
               fallback_ticks=sum(r["status"] != SAFE for r in records))
    if lat:
        out["latency_ms_p50"] = float(np.percentile(lat, 50))
        out["latency_ms_p99"] = float(np.percentile(lat, 99))
    return out

"""Per-tick records and the paper's run metrics (paper_1906_02318_gb300.metrics)
on hand-made ticks whose values are worked out here."""
import math

import numpy as np

from paper_1906_02318_gb300 import metrics


def _res(index, status, n_safe, u_r):
    return dict(index=index, status=status, n_safe=n_safe, u_r=np.asarray(u_r, dtype=float))


def test_tick_record_deviation_and_safe_fraction():
    # the user's input is safe: it is the selection and is not a sampled rollout
    r = metrics.tick_record(_res(0, metrics.SAFE, 41, [0.25]), [0.25], tick=3, trial=0,
                            n_samples=100, latency_s=1.5e-5)
    assert r["deviation"] == 0.0 and r["safe_fraction"] == 0.40
    assert math.isclose(r["latency_ms"], 0.015)
    # an intervention: distance 0.5 (3-4-5 scaled), every safe slot is a sample
    r = metrics.tick_record(_res(17, metrics.SAFE, 40, [0.1, 0.7]), [0.4, 0.3], tick=4,
                            trial=0, n_samples=100)
    assert math.isclose(r["deviation"], 0.5) and r["safe_fraction"] == 0.40
    # no safe candidate (fallback): the longest survivor is applied
    r = metrics.tick_record(_res(5, 1, 0, [-1.0]), [1.0], tick=5, trial=1, n_samples=100)
    assert r["deviation"] == 2.0 and r["safe_fraction"] == 0.0 and r["status"] == 1
    # the samples alone (Alg. 2 as printed): slot 0 is a sample
    r = metrics.tick_record(_res(0, metrics.SAFE, 10, [0.2]), [0.25], tick=6, trial=1,
                            n_samples=100, include_user=False)
    assert r["safe_fraction"] == 0.10 and math.isclose(r["deviation"], 0.05)


def test_summary_of_trials(tmp_path):
    recs = []
    # trial 0: 4 ticks, fails after the last; trial 1: 2 ticks, fails; trial 2: 3 ticks, safe
    for trial, n, fails in ((0, 4, True), (1, 2, True), (2, 3, False)):
        for k in range(n):
            recs.append(dict(tick=len(recs), trial=trial, status=metrics.SAFE, index=1, n_safe=5,
                             safe_fraction=0.1 * (k + 1), deviation=0.2 * trial,
                             latency_ms=1.0 + len(recs), failed=fails and k == n - 1))
    recs[2]["status"] = 1
    path = str(tmp_path / "ticks.jsonl")
    with metrics.TickLog(path) as log:
        for r in recs:
            log.write(r)
    back = metrics.read_log(path)
    assert back == recs
    s = metrics.summarize(back, tick_period_s=0.01)
    assert s["ticks"] == 9 and s["trials"] == 3
    assert math.isclose(s["safe_trial_fraction"], 1 / 3)
    assert math.isclose(s["mean_time_to_failure_s"], (0.04 + 0.02) / 2)
    dev = [0.0] * 4 + [0.2] * 2 + [0.4] * 3
    assert math.isclose(s["avg_deviation"], np.mean(dev))
    assert math.isclose(s["avg_deviation_std"], np.std(dev))
    sf = [0.1, 0.2, 0.3, 0.4, 0.1, 0.2, 0.1, 0.2, 0.3]
    assert math.isclose(s["avg_safe_rollouts"], np.mean(sf))
    assert s["fallback_ticks"] == 1
    assert math.isclose(s["latency_ms_p50"], 5.0)

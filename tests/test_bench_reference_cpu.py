"""The benchmark's reference arm (the FP64 oracle on the host cores) on CPU: a
run asked for more steps than fit its time budget stops once the budget of
timed work is spent and reports the steps it timed; its rate is per step.
The oracle's EM step is replaced by a fixed-duration stand-in so the test
takes a second."""
import json
import time
import types

import numpy as np


def test_reference_arm_stops_at_its_time_budget(monkeypatch, capsys):
    import bench
    import oracle

    step_s = 0.02
    calls = {"n": 0}

    def em_step(x, *a, **k):
        time.sleep(step_s)
        calls["n"] += 1
        return x

    nsub = 2
    monkeypatch.setattr(bench, "REF_BUDGET_S", 0.2)
    monkeypatch.setattr(oracle, "build", lambda: None)
    monkeypatch.setattr(oracle, "max_threads", lambda: 4)
    monkeypatch.setattr(oracle, "sensitivity", lambda *a, **k: np.ones((bench.NZ, bench.NX, bench.NX)))
    monkeypatch.setattr(oracle, "forward", lambda *a, **k: np.ones((nsub, bench.NZ, bench.NX)))
    monkeypatch.setattr(oracle, "em_step", em_step)
    args = types.SimpleNamespace(steps=1000, warmup=1, cpu_views=nsub)
    bench.run_reference(args)
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert out["impl"] == "reference" and out["steps_requested"] == 1000
    # the budget allows about 0.2 / 0.02 = 10 timed steps, never the 1000 asked for
    assert 3 <= out["steps"] <= 12, out["steps"]
    assert calls["n"] == out["steps"] + 1  # plus the one warm-up step
    # ms_per_step is the measured time of one timed step (steps x ms_per_step fits the run); the rate is
    # steps x (views sampled / 128) per second of timed work
    per_step = out["ms_per_step"] / 1e3
    assert abs(per_step - step_s) < 0.5 * step_s
    assert out["steps"] * per_step < 2 * bench.REF_BUDGET_S
    assert abs(out["value"] - (nsub / 128) / per_step) < 1e-9 * out["value"]
    assert abs(out["extrapolated_ms_per_pair"] - out["ms_per_step"] * 128 / nsub) < 1e-9 * out["ms_per_step"]
    assert out["e2e"]["value"] == out["value"] and out["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_samples_one_view_per_host_thread(monkeypatch, capsys):
    """The oracle's parallel axis is the views: the default sample gives every host thread one view, so the
    cores the line reports are the cores the oracle used."""
    import bench
    import oracle

    seen = {}

    def em_step(x, y, *a, **k):
        seen["views"] = y.shape[0]
        return x

    monkeypatch.setattr(oracle, "build", lambda: None)
    monkeypatch.setattr(oracle, "max_threads", lambda: 12)
    monkeypatch.setattr(oracle, "sensitivity", lambda *a, **k: np.ones((bench.NZ, bench.NX, bench.NX)))
    monkeypatch.setattr(oracle, "forward", lambda *a, **k: np.ones((12, bench.NZ, bench.NX)))
    monkeypatch.setattr(oracle, "em_step", em_step)
    bench.run_reference(types.SimpleNamespace(steps=1, warmup=0, cpu_views=0))
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert seen["views"] == 12 and out["cpu_baseline"]["cores"] == 12

"""The benchmark's reference arm (the FP64 oracle on the host cores) runs without a GPU and
prints one JSON line with the keys the benchmark contract asks for."""
import contextlib
import io
import json
import types

import bench


import pytest


@pytest.mark.parametrize("workload", ["cone3d_512", "fan2d_512"])
def test_reference_arm_json(monkeypatch, workload):
    leg = bench.cpu_oracle_leg
    monkeypatch.setattr(bench, "cpu_oracle_leg", lambda steps, target_s=15.0: leg(steps, target_s=1.0))
    monkeypatch.setattr(bench, "REFERENCE_TOTAL_S", 1.5)
    args = types.SimpleNamespace(steps=2, warmup=1, workload=workload)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args, 0, 1)
    line = json.loads(out.getvalue().strip().splitlines()[-1])
    assert line["config"]["workload"].startswith(workload)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(types.SimpleNamespace(steps=1, warmup=0), 1, 2)
    assert out.getvalue() == ""

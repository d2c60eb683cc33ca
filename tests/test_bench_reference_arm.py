"""The bench's reference arm on CPU: the oracle as it stands, timed on a bounded sample, printed as one
JSON line with the keys the bench contract asks for."""
import json

import pytest


def test_reference_arm_prints_one_contract_line(capsys):
    import bench

    class Args:
        workload = bench.DEFAULT_WORKLOAD
        steps = 1
        warmup = 0
        ref_iterations = 2706
        loads = "traction"
        blocks = "vertex"
        eta_bar = 1.0

    assert bench.run_reference(Args, 0, 1) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1 and d["steps"] == 1
    # value: the workload's time-to-solution scaled from the sample; ms_per_step: what the sample took
    assert d["value"] > 0 and 0 < d["ms_per_step"] < 120e3 and d["value"] * 1e3 > d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and "window" in cb["sample"]
    # a complete oracle solve of a small member of the family, measured, not scaled
    fs = cb["full_solve_measured"]
    assert fs["oracle_solve_s"] > 0 and fs["oracle_iterations"] > 10 and fs["oracle_threads"] == 1
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

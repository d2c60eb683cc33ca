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
        ref_iterations = 877
        loads = "traction"
        blocks = "vertex"
        eta_bar = 1.0

    assert bench.run_reference(Args, 0, 1) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "s"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] == pytest.approx(d["value"] * 1e3)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and "window" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

"""bench.py's reference arm on the host: the FP64 oracle timed on the host cores prints
the same one-line JSON record as the GPU arm (metric, unit, steps, config, cpu_baseline,
e2e), with "impl": "reference".  No GPU is needed for it."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--config", "grid33"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["metric"] == bench.METRIC
    assert rec["unit"] == "evals/s" and rec["higher_is_better"] is True and rec["value"] > 0
    assert rec["steps"] == 1 and rec["warmup"] == 0 and rec["n_gpus"] == 1
    assert rec["ms_per_step"] == pytest.approx(1e3 * rec["config"]["batch"] / rec["value"], rel=1e-9)
    base = rec["cpu_baseline"]
    assert base["kind"] == "oracle" and base["value"] == rec["value"] and base["cores"] >= 1
    assert rec["e2e"] == {"value": rec["value"], "unit": "evals/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert rec["config"]["workload"].startswith("grid33")

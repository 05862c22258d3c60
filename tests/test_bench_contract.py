"""The JSON line bench.py prints: the keys and types the benchmark contract
requires, for the reference arm (the oracle on the CPU, no GPU) and for the
GPU arm on a quick run."""
import contextlib
import io
import json

import pytest

import bench

BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
             "cpu_baseline"}


def _run(argv):
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.main(argv)
    lines = [line for line in out.getvalue().splitlines() if line.startswith("{")]
    assert len(lines) == 1, out.getvalue()
    return json.loads(lines[0])


def _check_common(d):
    assert BASE_KEYS <= set(d), BASE_KEYS - set(d)
    assert d["unit"] == "mults/s" and d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["warmup"] >= 3
    assert "workload" in d["config"] and "model" not in d["config"]
    e2e = d["e2e"]
    assert {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"} <= set(e2e)
    cpu = d["cpu_baseline"]
    assert {"value", "unit", "cores", "kind", "sample"} <= set(cpu) and cpu["kind"] == "oracle"


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-step-budget", "0.2",
              "--quick"])
    _check_common(d)
    assert d["impl"] == "reference"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] == d["cpu_baseline"]["value"]


def test_warmup_below_three_is_refused():
    with pytest.raises(SystemExit):
        bench.main(["--warmup", "2"])


@pytest.mark.gpu
def test_gpu_arm_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--quick", "--steps", "2", "--warmup", "3", "--e2e-steps", "1", "--cpu-budget", "0.5",
              "--mixed-items", "2000", "--mixed-steps", "1", "--serve-requests", "0",
              "--fused-reps", "1", "--isolated-reps", "1"])
    _check_common(d)
    assert d["impl"] == "ours" and d["n_gpus"] == 1
    roof = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(roof)
    assert roof["bound"] in ("hbm", "tensor", "alu") and 0 < roof["frac"] < 2
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["gpu_launches"] == 2 * len(d["config"]["ops_per_step"])
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["mixed"]["results_identical"] is True

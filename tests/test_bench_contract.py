"""The JSON line bench.py prints: the keys and types the benchmark contract
requires, for the reference arm (the oracle on the CPU, no GPU) and for the
GPU arm on a quick run; the line stays short enough to parse whole, and the
reference arm's step time is the time it measured."""
import contextlib
import io
import json
import time

import pytest

import bench

MAX_LINE = 3000

BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
             "cpu_baseline"}


def _run(argv):
    out, err = io.StringIO(), io.StringIO()
    with contextlib.redirect_stdout(out), contextlib.redirect_stderr(err):
        bench.main(argv)
    lines = [line for line in out.getvalue().splitlines() if line.startswith("{")]
    assert len(lines) == 1, out.getvalue()
    assert len(lines[0]) <= MAX_LINE, len(lines[0])
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
    t = time.perf_counter()
    d = _run(["--impl", "reference", "--steps", "2", "--warmup", "3", "--ref-step-budget", "0.2",
              "--quick"])
    wall = time.perf_counter() - t
    _check_common(d)
    assert d["impl"] == "reference"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] == d["cpu_baseline"]["value"]
    # the steps it claims ran inside this call: no extrapolated step time
    assert d["ms_per_step"] * d["steps"] / 1e3 <= d["timed_s"] + 1e-3 <= wall + 1e-3
    assert d["extrapolated_full_step_s"] * 1e3 >= d["ms_per_step"]


def test_reference_arm_full_line_is_short():
    """The default (all 33 ops) reference line, on a tiny sample."""
    d = _run(["--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-step-budget", "0.05"])
    assert d["config"]["ops_per_step"] == 33


def test_compact_line_of_a_full_record():
    """A full GPU-arm record with every section (33 ops, all forms at 9
    sizes, mixed and serving runs) compacts to a short line carrying the
    contract's keys and the summary figures."""
    ops = bench.build_ops()
    roof = [{"op": o.label, "bound": "alu", "achieved": 1.234, "peak": 6.712,
             "unit": "T word-products/s", "frac": 0.1839, "peak_kind": "x" * 120, "traffic": None}
            for o in ops]
    full = {"metric": bench.METRIC, "value": 2.7e7, "unit": "mults/s", "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 44.7, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": bench.workload_config(ops, 1), "impl": "ours", "add_gbs": 5300.1,
            "roofline": dict(roof[-3], traffic=588000000, kernel_share_of_step=0.08, ms=3.5),
            "rooflines": roof, "breakdown": [{"op": o.label, "ms": 1.0} for o in ops],
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "sm_mhz_min": 2070.0,
                       "power_w_max": 900.0, "reasons": [], "samples": 400},
            "gpu_launches": 660, "skipped_ops": [],
            "e2e": {"value": 2.3e7, "unit": "mults/s", "h2d_bytes_per_step": 8_300_000_000,
                    "d2h_bytes_per_step": 4_000_000_000, "steps": 5, "ms_per_step": 50.0,
                    "ranks": 1, "api": "y" * 100},
            "cpu_baseline": {"value": 78000.0, "unit": "mults/s", "cores": 16, "kind": "oracle",
                             "sample": bench.sample_text(ops, {o.label: 410 for o in ops}, 0.2),
                             "sample_s": 15.0, "extrapolated_full_step_s": 70.0},
            "forms": {"crossover_bits": {"ntt64": 65536, "crt": 32768, "ntt3": 8192},
                      "ops": [{"op": "x@1K", "ms": 1.0}] * 54, "table_ms": {}},
            "mixed": {f: {"ms": 10.0} for f in ("batched", "plain_class", "plain_item")},
            "serving": {"runs": [{"mode": m, "offered_per_s": r, "throughput_per_s": 1.0,
                                  "p50_us": 1.0, "p99_us": 2.0}
                                 for m, r in (("batched", 50000), ("batched", 500000),
                                              ("sequential", 5000))]},
            "fused": {"sizes": [{"add6_over_add": 1.1, "poly_over_mul_low": 4.0}]}}
    full["mixed"].update(speedup_vs_class=2.0, speedup_vs_item=200.0, results_identical=True)
    line = json.dumps(bench.compact(full))
    assert len(line) <= MAX_LINE, len(line)
    d = json.loads(line)
    _check_common(d)
    assert d["frac"]["ntt64@256K"] == 0.1839 and len(d["frac"]) == len(bench.KEY_OPS)
    assert d["crossover_bits"]["ntt3"] == 8192
    assert d["mixed"]["speedup_vs_class"] == 2.0 and d["mixed"]["results_identical"] is True
    assert d["roofline"]["traffic"] == 588000000


def test_crossover_rule():
    t = {1024: {"quad": 1, "quadtc": 5, "ntt3": 2}, 2048: {"quad": 2, "quadtc": 3, "ntt3": 1},
         4096: {"quad": 4, "quadtc": 3, "ntt3": 2.5}, 8192: {"quad": 8, "quadtc": 4, "ntt3": 3}}
    assert bench.crossover_bits(t, "ntt3") == 2048
    t[4096]["ntt3"] = 3.5          # slower again at 4K: the crossover moves up
    assert bench.crossover_bits(t, "ntt3") == 8192
    t[8192]["ntt3"] = 9            # slower at the largest size: no crossover
    assert bench.crossover_bits(t, "ntt3") is None


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
              "--fused-reps", "1", "--isolated-reps", "1", "--seq-rate", "2000"])
    _check_common(d)
    assert d["impl"] == "ours" and d["n_gpus"] == 1
    roof = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(roof)
    assert roof["bound"] in ("hbm", "tensor", "alu") and 0 < roof["frac"] < 2
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["gpu_launches"] == 2 * d["config"]["ops_per_step"]
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert d["mixed"]["results_identical"] is True
    assert set(d["crossover_bits"]) == {"ntt64", "crt", "ntt3"}

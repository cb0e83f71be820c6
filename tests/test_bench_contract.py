"""bench.py's output contract on the CPU: the reference arm (the oracle) prints
one JSON line with every key the contract names, and the roofline helper's
arithmetic and traffic guard (no GPU)."""
import json
import os
import subprocess
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def test_reference_arm_prints_one_contract_line():
    # run in a process that afterwards checks it never loaded the CUDA path
    code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--L', '5', '--steps', '2', "
            "'--warmup', '3']; runpy.run_path('bench.py', run_name='__main__'); "
            "maps = open('/proc/self/maps').read(); "
            "assert 'libhwfv1' not in maps and 'paper_2206_05761_gb300' not in sys.modules, 'CUDA path loaded'")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and KEYS <= set(d)
    assert d["value"] > 0 and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == "terrain_flood" and d["config"]["L"] == 5
    assert d["warmup"] == 3 and d["steps"] == 2
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host_cores"] == os.cpu_count()
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_roofline_of_the_wet_leaf_update(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    args = types.SimpleNamespace(precision=64)
    r = {"kernels_ms": {"k_fv1_faces": 0.04, "k_fv1_update": 0.03}, "update_ms": 0.066,
         "wet_per_step": 74000.0}
    roof = bench.roofline("k_fv1_faces", 0.04, r, args, {"hbm_gbs": 6699.8}, "measured")
    # 294 FLOP per wet leaf over the update's in-step time, against the FP64 pipe
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert abs(roof["achieved"] - 294 * 74000.0 / 66e-6 / 1e12) < 1e-12
    assert abs(roof["peak"] - 152 * 2 * 2.07e9 / 1e12) < 1e-12
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-15
    # the ncu traffic is reported only while the kernel source is the one it was taken on
    monkeypatch.setattr(bench, "kernels_sha256", lambda: bench.FV1_WET_TRAFFIC["kernels_sha256"])
    assert bench.roofline("k_fv1_faces", 0.04, r, args, {}, "")["traffic"] == \
        bench.FV1_WET_TRAFFIC["bytes_per_launch"]
    monkeypatch.setattr(bench, "kernels_sha256", lambda: "0" * 64)
    assert bench.roofline("k_fv1_faces", 0.04, r, args, {}, "")["traffic"] is None

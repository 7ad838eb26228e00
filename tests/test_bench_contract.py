"""The benchmark's reference arm (the oracle on the host cores) runs without
a GPU: its JSON line carries the keys the benchmark contract asks for, with
the same metric, unit and direction as the GPU arm, an e2e object without
host-device traffic and a cpu_baseline describing the run."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--grid", "20"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [l for l in out.stdout.splitlines() if l.strip().startswith("{")][-1]
    d = json.loads(line)
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["vs_baseline"] is None and d["scaling"] == "weak"
    assert isinstance(d["config"], dict) and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_weighted_roofline_is_the_launch_weighted_mix():
    """The roofline weights each width by its launches: achieved = sum of
    launches x bytes over sum of launches x time of the dominant kernel; the
    traffic is reported only when every width has a profile."""
    sys.path.insert(0, ROOT)
    import bench
    per = {"factor_spmv": {"rows": [
               {"k": 1, "complex": True, "launches": 300, "ms": 0.02, "bytes": 100e6, "GBs": 5000.0, "traffic": 90e6},
               {"k": 7, "complex": True, "launches": 100, "ms": 0.06, "bytes": 200e6, "GBs": 3333.3, "traffic": 210e6}]},
           "op_spmv": {"rows": [
               {"k": 7, "complex": True, "launches": 20, "ms": 0.09, "bytes": 230e6, "GBs": 2555.6, "traffic": None}]}}
    roof, other = bench.weighted_roofline(per, 6000.0)
    assert roof["kernel"] == "factor_spmv"
    t = 300 * 0.02 + 100 * 0.06
    b = 300 * 100e6 + 100 * 200e6
    assert abs(roof["achieved"] - b / (t * 1e-3) / 1e9) < 1e-9
    assert abs(roof["frac"] - roof["achieved"] / 6000.0) < 1e-12
    assert abs(roof["traffic"] - (300 * 90e6 + 100 * 210e6) / 400) < 1.0
    assert roof["algorithmic_bytes_per_launch"] == int(b / 400)
    assert abs(other["factor_spmv"]["share_of_spmv_time"] - t / (t + 20 * 0.09)) < 1e-12
    per["factor_spmv"]["rows"][1]["traffic"] = None
    assert bench.weighted_roofline(per, 6000.0)[0]["traffic"] is None


def test_spmv_bytes_by_layout():
    """Algorithmic bytes of one SpMV launch: CSR counts its column indices and
    row pointers, the diagonal layout has none (and its padding is not
    counted); the vectors are the same in both."""
    sys.path.insert(0, ROOT)
    import bench
    n, nnz, k = 1000, 6900, 6
    for kern, vec in (("factor_spmv", 2), ("op_spmv", 3)):
        csr = bench._spmv_bytes(kern, k, n, nnz, True, True, bench.FORMATS["csr"])
        dia = bench._spmv_bytes(kern, k, n, nnz, True, True, bench.FORMATS["dia"])
        assert csr - dia == nnz * 4 + 4 * (n + 1)
        vals = nnz * (8 if kern == "factor_spmv" else 4) + (4 * n if kern == "op_spmv" else 0)
        assert dia == vals + vec * k * n * 8
    assert bench.FORMAT_NAMES[bench.FORMATS["dia"]] == "dia"

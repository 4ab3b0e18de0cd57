"""bench.py's output contract, checked without a GPU: the reference arm (the oracle timed on the
host) prints one JSON line with the keys the bench contract names, and the per-launch DRAM
traffic is only reported for the kernel sources it was captured on."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_traffic_is_reported_only_for_the_captured_sources():
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_sources_sha256()
    assert h == bench.kernel_sources_sha256() and len(h) == 64
    saved = dict(bench.TRAFFIC)
    try:
        bench.TRAFFIC[("fp64", "dataflow")] = {"bytes_per_launch": 123, "capture": "c1", "sources_sha256": h}
        assert bench.traffic_for("fp64", "dataflow") == (123, "c1")
        assert bench.traffic_for("fp64", "levels") == (None, None)
        bench.TRAFFIC[("fp64", "dataflow")] = {"bytes_per_launch": 123, "capture": "c1", "sources_sha256": "0" * 64}
        assert bench.traffic_for("fp64", "dataflow") == (None, None)
    finally:
        bench.TRAFFIC.clear()
        bench.TRAFFIC.update(saved)


def test_roofline_work_per_update_is_the_methods():
    """The fractions use the method's algorithmic work per update (assembly, inflow faces, LU,
    solves), the same figure for every arithmetic form; the double-single form's issued FP32 flops
    (its emulation of wider arithmetic) are reported separately and are larger."""
    sys.path.insert(0, ROOT)
    import bench
    w = bench.alg_work(2, 3)
    assert w["flops"] == 5800.0 and w["bytes"] == 350.0
    assert bench.alg_work(3, 2)["flops"] == 35000.0
    assert bench.ds_fp32_issued_flops_per_update(2, 3, 2) > 2 * w["flops"]


def test_stored_inverse_bytes_per_update():
    """8 (N^2 + F blk + 2N) bytes per update: the inverse, F inflow blocks (2D folded N x Nf,
    3D Nf x Nf), the flux written and about N entries of traces and source.  F is the average
    number of inflow faces: dim for quadrilaterals and hexahedra; for a flat-faced simplex the
    scaled normals sum to zero, so over directions half its faces are inflow (1.5 of 3, 2 of 4)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.inv_alg_bytes(2, 3) == 8 * (16 * 16 + 2 * 16 * 4 + 2 * 16) == 3328
    assert bench.inv_alg_bytes(3, 2) == 8 * (27 * 27 + 3 * 9 * 9 + 2 * 27) == 8208
    assert bench.inv_alg_bytes(2, 3, simplex=True) == 8 * (10 * 10 + 1.5 * 10 * 4 + 2 * 10) == 1440
    assert bench.inv_alg_bytes(3, 2, simplex=True) == 8 * (10 * 10 + 2 * 6 * 6 + 2 * 10) == 1536
    assert bench.inv_alg_bytes(3, 1, simplex=True) == 8 * (4 * 4 + 2 * 3 * 3 + 2 * 4)

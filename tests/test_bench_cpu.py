"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle timed on
the host) and the helpers the GPU arm uses to name kernels and read the
committed DRAM-traffic record."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "64",
                          "--steps", "3", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["grid"] == [64, 64] and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_nothing_on_other_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--size", "64",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                         env=env)
    assert out.returncode == 0, out.stderr
    assert not [x for x in out.stdout.splitlines() if x.startswith("{")]


@pytest.mark.parametrize("n,row,col", [
    (256, "row_kernel<256,ROW_PT>", "col_kernel<256,COL_T>"),
    (512, "row_pair_kernel<512>", "col_kernel<512,COL_T>"),
    (1024, "row_pair_kernel<1024>", "col_pair_kernel<1024,COL_T>"),
    (2048, "row_pair_kernel<2048>", "col_pair_kernel<2048,COL_T>"),
    (4096, "row_pair_kernel<4096>", "col_pair_kernel<4096,COL_T>"),
    (8192, "row_pair_kernel<8192>", "col_pair_kernel<8192,COL_T>")])
def test_kernel_names_follow_the_pass_dispatch(n, row, col):
    import bench
    assert bench.row_kernel_name(n) == row
    assert bench.col_kernel_name(n) == col


def test_traffic_record_is_keyed_by_the_kernel_sources():
    import bench
    h = bench.kernel_source_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    rows = [dict(x.split("=", 1) for x in line.split() if "=" in x) for line in open(path)
            if line.strip() and not line.startswith("#")]
    assert rows
    for kv in rows:
        assert {"kernel", "grid", "src", "dram_bytes_per_launch"} <= set(kv)
        assert float(kv["dram_bytes_per_launch"]) > 0
        got = bench.recorded_traffic(kv["kernel"], int(kv["grid"].split("x")[0]))
        # a record is only used while the sources it was taken on are unchanged
        assert (got is not None) == (kv["src"] == h)

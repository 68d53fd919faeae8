"""bench.py's reference arm (the CPU oracle, as it stands) prints the contract's
JSON line on a small case, on the same metric, unit, workload and config block
as the GPU arm, timing the step's own algorithm on every host core (no GPU
needed)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# what the sample description must name for each solver
ALGORITHM = {"mg": "multigrid", "ssor": "SSOR", "mixed": "Jacobi-PCG", "pif": "direct-sum"}


@pytest.mark.parametrize("solver", ["mg", "ssor", "mixed", "pif"])
def test_reference_arm_json_line(solver):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--N", "16", "--ppc", "2",
                          "--steps", "1", "--warmup", "0", "--solver", solver], cwd=ROOT, capture_output=True,
                         text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert r["impl"] == "reference" and "unavailable" not in r
    assert r["metric"] == bench.METRIC and r["unit"] == bench.UNIT and r["higher_is_better"] is True
    assert r["value"] > 0 and r["steps"] == 1 and r["warmup"] == 0
    args = bench.parse(["--N", "16", "--ppc", "2", "--solver", solver])
    assert r["config"] == bench.pic_config(args, 1)
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == r["value"] and cb["sample"]
    assert cb["cores"] == os.cpu_count() and cb["cores"] >= 1
    assert ALGORITHM[solver] in cb["sample"], cb["sample"]
    if solver != "pif":
        assert "warm-started" in cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}

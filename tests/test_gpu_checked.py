"""The bounds-checked build (every derived node coordinate tested before it
indexes memory; faults recorded in a device word, never trapped): all kernel
families on ragged grids with every wall combination record no fault and still
match the FP64 oracle."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_records_no_index_fault():
    env = dict(os.environ, LBM_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked", "run_checked.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] == 1
    assert len(out["faults"]) > 30 and all(f == 0 for f in out["faults"]), out["faults"]
    assert out["max_rel"] <= 1e-5

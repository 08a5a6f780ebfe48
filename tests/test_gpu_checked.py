"""The bounds-checked build of the library (-DDPC_CHECKED, a stand-in for a
memory checker): built here, it gives every application at every level the
oracle's results with status 0, and turns an out-of-range column index into
DPC_ERR_OVERFLOW instead of a memory access outside the arrays."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu


def test_checked_build_exact_and_reports_bad_indices():
    from paper_1606_08150_gb300 import build

    lib = build.build(checked=True)
    assert os.path.exists(lib) and lib != build.LIB
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "checked_child.py")
    out = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=900,
                         env=dict(os.environ, DPC_LIBRARY="checked"))
    assert out.returncode == 0, out.stderr[-3000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["checked"], res["library"]
    good = [c for c in res["cases"] if "ok" in c]
    assert len(good) >= 50
    bad_results = [c for c in good if not c["ok"] or c["status"] != 0]
    assert not bad_results, bad_results
    malformed = [c for c in res["cases"] if "ok" not in c]
    assert len(malformed) == 12
    assert all(c["status"] == 6 for c in malformed), malformed  # DPC_ERR_OVERFLOW

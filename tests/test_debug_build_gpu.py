"""The index-checked debug build (-DSHT_DEBUG): every kernel checks its tile,
stage, tensor-memory, shared-memory and global offsets and counts violations
instead of touching memory outside a buffer.  A child process runs every form
and launch path of the library once on small grids through that build; no
check may fire and every result must still match the oracle.  The release
library reports that it was built without the checks."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_runs_every_path_without_a_violation():
    from paper_1010_1260_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, SHT_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join("tests", "_debug_child.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert out["library"] == lib
    for name, rep in out["reports"].items():
        assert rep["checks_built"], name
        assert rep["violations"] == 0, (name, rep)
    for key, err in out["errors"].items():
        tol = 1e-10 if key.endswith(("fp64", "adjoint", "partitioned")) or "/fp64/" in key else (
            1e-5 if "fp32_tc" in key else 1e-6)
        assert err < tol, (key, err)


def test_release_build_has_no_checks():
    from paper_1010_1260_gb300 import sht
    plan = sht.Plan(sht.healpix(4), 8)
    rep = plan.debug_report()
    assert not rep["checks_built"] and rep["violations"] == 0
